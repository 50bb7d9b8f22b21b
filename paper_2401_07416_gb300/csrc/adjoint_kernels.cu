// Reverse-time kernels of the adjoint (gradient of a loss of the time-integrated
// detector flux) and the chain rule from dL/dV to the atom parameters.
//
// Forward step n -> n+1 (Sec. 2.1, Eqs. 8-9, with the absorbing factor M and the
// detector flux j): It = I + A R; j = cj (R_kd It_kd+1 - R_kd+1 It_kd);
// Rt = R - A It; R' = M Rt; I' = M It.  A is symmetric, so one backward step,
// with (P, Q) the adjoints of (R', I') and w = dL/dF * dt * cj per pixel, is
//   a. It = I'/M, Rt = R'/M, Pt = M P                         (per plane)
//   b. R = Rt + A It,  Qt = M Q - A Pt                        (undo Eq. 8; adjoint of Eq. 8)
//   c. Qt[kd+1] += w R[kd],  Qt[kd] -= w R[kd+1]              (flux w.r.t. It)
//   d. gV -= cv (Qt R - Pt It);  P = Pt + A Qt + dj/dR        (adjoint of Eq. 9, V terms)
//   e. I = It - A R,  Q = Qt                                  (undo Eq. 9)
// after which (R, I) = (R^n, I^{n-1/2}) and (P, Q) their adjoints.  Step a is not a
// pass of its own, and d and e share one: the kernels scale what they read by the plane's
// factor (M, or its reciprocal, in the context's number format: the forward
// multiplied by exactly that M; 1 outside the absorbing layers).  FP32 contexts
// form every product, including the dL/dV term, in FP32 and only accumulate gV in
// FP64.  Arrays are unpadded [nz][ny][nx]; neighbours wrap on periodic axes and read
// zero on walls.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "tdse_internal.cuh"

namespace tdse {
namespace {

constexpr int kThreads = 256;

struct Geo {
    int nx, ny, nz;
    int per[3];
    double cx, cy, cz, cv, c0;   // c0 = -2 (cx + cy + cz)
    long long pitch, pplane;     // strides of the forward's padded arrays (d)
    int G;                       // their ghost width
};

__device__ __forceinline__ long long cell(const Geo &g, int x, int y, int z)
{
    return (static_cast<long long>(z) * g.ny + y) * g.nx + x;
}

// Each thread of the step kernels below updates kCells consecutive x-cells (nx is a
// multiple of 4) with 16-byte accesses: four independent cells per thread instead of
// one, and no pointer aliasing between the fields.
constexpr int kCells = 4;

template <typename Real>
__device__ __forceinline__ void ld4(const Real *__restrict__ p, Real (&v)[kCells])
{
    if constexpr (sizeof(Real) == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const double2 a = reinterpret_cast<const double2 *>(p)[0];
        const double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
}

template <typename Real>
__device__ __forceinline__ void st4(Real *__restrict__ p, const Real (&v)[kCells])
{
    if constexpr (sizeof(Real) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
}

// The kCells values of row (y, z) at x0.. of f, with y and z at most one cell outside
// the grid: the periodic image (one wrap) or zeros beyond a wall.
template <typename Real>
__device__ __forceinline__ void row4(const Real *__restrict__ f, const Geo &g, int x0, int y, int z,
                                     Real (&v)[kCells])
{
    bool zero = false;
    if (y < 0 || y >= g.ny) {
        if (g.per[1]) y += y < 0 ? g.ny : -g.ny;
        else zero = true;
    }
    if (z < 0 || z >= g.nz) {
        if (g.per[2]) z += z < 0 ? g.nz : -g.nz;
        else zero = true;
    }
    if (zero) {
#pragma unroll
        for (int k = 0; k < kCells; ++k) v[k] = Real(0);
        return;
    }
    ld4(f + cell(g, x0, y, z), v);
}

// d = -2 (cx + cy + cz) - cv V at the kCells cells, read from the forward step's own
// array so that the reconstruction undoes exactly the forward's arithmetic.
template <typename Real>
__device__ __forceinline__ void dval4(const Real *__restrict__ D, const Geo &g, int x0, int y, int z,
                                      Real (&d)[kCells])
{
    ld4(D + static_cast<long long>(z) * g.pplane + static_cast<long long>(y + g.G) * g.pitch + (x0 + g.G), d);
}

// Plane z's factor sc[z] for z at most one plane outside the grid: wrapped on a
// periodic axis, any value beyond a wall (the neighbour reads zero there).
template <typename Real>
__device__ __forceinline__ Real plane_factor(const Real *__restrict__ sc, const Geo &g, int z)
{
    if (z < 0 || z >= g.nz) {
        if (!g.per[2]) return Real(1);
        z += z < 0 ? g.nz : -g.nz;
    }
    return sc[z];
}

// Rounded products the compiler may not fuse into a following add: the three-pass
// and the fused step must round every operation identically.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

// A f at one cell from its (already scaled) operands: cx (f[x+1] + f[x-1]) + cy (..) +
// cz (..) + d f as one FMA chain.  Both the three-pass and the fused backward step
// use this, and the explicit updates below, so they round identically.
template <typename Real>
__device__ __forceinline__ Real stencil(const Geo &g, Real xm, Real xp, Real ym, Real yp, Real zm,
                                        Real zp, Real c, Real d)
{
    return fma(static_cast<Real>(g.cx), xp + xm,
               fma(static_cast<Real>(g.cy), yp + ym, fma(static_cast<Real>(g.cz), zp + zm, rmul(d, c))));
}

// out = A (s f) at the kCells cells (x0 + k, y, z), cell offset o of x0; s a per-plane
// factor (NULL: 1).  Per cell: every operand scaled by its plane's factor, then
// cx (f[x+1] + f[x-1]) + cy (..) + cz (..) + d f as one FMA chain.
template <typename Real>
__device__ __forceinline__ void apply_A4(const Real *__restrict__ f, const Real (&d)[kCells],
                                         const Geo &g, int x0, int y, int z, long long o,
                                         const Real *__restrict__ sc, Real (&out)[kCells])
{
    Real c[kCells], ym[kCells], yp[kCells], zm[kCells], zp[kCells];
    ld4(f + o, c);
    row4(f, g, x0, y - 1, z, ym);
    row4(f, g, x0, y + 1, z, yp);
    row4(f, g, x0, y, z - 1, zm);
    row4(f, g, x0, y, z + 1, zp);
    Real xl, xr;   // the x-neighbours of the group
    if (x0 > 0) xl = f[o - 1];
    else xl = g.per[0] ? f[o - 1 + g.nx] : Real(0);
    if (x0 + kCells < g.nx) xr = f[o + kCells];
    else xr = g.per[0] ? f[o + kCells - g.nx] : Real(0);
    Real s0 = Real(1), sm = Real(1), sp = Real(1);
    if (sc) {
        s0 = sc[z];
        sm = plane_factor(sc, g, z - 1);
        sp = plane_factor(sc, g, z + 1);
    }
#pragma unroll
    for (int k = 0; k < kCells; ++k) {
        Real xm = k == 0 ? xl : c[k - 1];
        Real xp = k == kCells - 1 ? xr : c[k + 1];
        Real y0 = ym[k], y1 = yp[k], z0 = zm[k], z1 = zp[k], cc = c[k];
        if (sc) {
            xm = rmul(xm, s0);
            xp = rmul(xp, s0);
            y0 = rmul(y0, s0);
            y1 = rmul(y1, s0);
            cc = rmul(cc, s0);
            z0 = rmul(z0, sm);
            z1 = rmul(z1, sp);
        }
        out[k] = stencil(g, xm, xp, y0, y1, z0, z1, cc, d[k]);
    }
}

// The step kernels below run a 2-D grid: blockIdx.x * blockDim.x + threadIdx.x
// is the group of kCells cells (x0.., y) of a plane (32-bit index arithmetic), the
// planes are blockIdx.y, blockIdx.y + gridDim.y, ...

#define GRID_STRIDE(t, n)                                                                     \
    for (long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; t < (n); \
         t += static_cast<long long>(gridDim.x) * blockDim.x)

// b. R = Rt + A It (undo Eq. 8), Qt = M Q - A Pt (adjoint of Eq. 8); Mk is M per
// plane, Mi its reciprocal
template <typename Real>
__global__ void adj_b_kernel(Geo g, const Real *__restrict__ Mk, const Real *__restrict__ Mi,
                             const Real *__restrict__ D, Real *__restrict__ R,
                             const Real *__restrict__ I, const Real *__restrict__ P,
                             Real *__restrict__ Q)
{
    const int gx = g.nx / kCells;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gx * g.ny) return;
    const int x0 = (t % gx) * kCells, y = t / gx;
    for (int z = blockIdx.y; z < g.nz; z += gridDim.y) {
        const long long o = cell(g, x0, y, z);
        Real d[kCells], r[kCells], q[kCells], ai[kCells], ap[kCells];
        dval4(D, g, x0, y, z, d);
        ld4(R + o, r);
        ld4(Q + o, q);
        apply_A4(I, d, g, x0, y, z, o, Mi, ai);
        apply_A4(P, d, g, x0, y, z, o, Mk, ap);
        const Real mi = Mi[z], mk = Mk[z];
#pragma unroll
        for (int k = 0; k < kCells; ++k) {
            r[k] = fma(r[k], mi, ai[k]);
            q[k] = fma(q[k], mk, -ap[k]);
        }
        st4(R + o, r);
        st4(Q + o, q);
    }
}

// c. the detector flux w.r.t. It; also keeps It of the two detector planes (Ist[0..plane)
// = plane kd, Ist[plane..2 plane) = plane kd+1) for dj/dR in the pass below, which
// overwrites I
template <typename Real>
__global__ void adj_flux_q_kernel(Geo g, int kd, const double *__restrict__ w,
                                  const Real *__restrict__ Mi, const Real *R,
                                  const Real *__restrict__ I, Real *Q, Real *__restrict__ Ist)
{
    const long long plane = static_cast<long long>(g.nx) * g.ny;
    GRID_STRIDE(p, plane)
    {
        const Real wp = static_cast<Real>(w[p]);
        Ist[p] = rmul(I[kd * plane + p], Mi[kd]);
        Ist[plane + p] = rmul(I[(kd + 1) * plane + p], Mi[kd + 1]);
        Q[(kd + 1) * plane + p] = fma(wp, R[kd * plane + p], Q[(kd + 1) * plane + p]);
        Q[kd * plane + p] = fma(-wp, R[(kd + 1) * plane + p], Q[kd * plane + p]);
    }
}

// Steps d and e at one cell: Pt = M P, It = I' / M, gV -= cv (Qt R - Pt It),
// P = Pt + A Qt (before the detector terms), I = It - A R.
template <typename Real>
__device__ __forceinline__ void de_cell(const Geo &g, Real p, Real i, Real qt, Real r, Real mk,
                                        Real mi, Real aq, Real ar, double &gv, Real &pn, Real &in)
{
    const Real pt = rmul(p, mk);
    const Real it = rmul(i, mi);
    const Real ptit = rmul(pt, it);
    gv = fma(-g.cv, static_cast<double>(fma(qt, r, -ptit)), gv);
    pn = pt + aq;
    in = it - ar;
}

// d and e in one pass, with Pt = M P and It = I' / M at the plane:
//   gV -= cv (Qt R - Pt It), P = Pt + A Qt + dj/dR   (adjoint of Eq. 9)
//   I = It - A R                                      (undo Eq. 9)
// Neither reads as a stencil what the other writes (Q and R are read, P and I written
// at the cell itself); dj/dR reads It of the other detector plane from Ist.
template <typename Real>
__global__ void adj_de_kernel(Geo g, const Real *__restrict__ Mk, const Real *__restrict__ Mi,
                              const Real *__restrict__ D, int kd, const double *__restrict__ w,
                              const Real *__restrict__ Ist, const Real *__restrict__ R,
                              Real *__restrict__ I, Real *__restrict__ P,
                              const Real *__restrict__ Q, double *__restrict__ gV)
{
    const long long plane = static_cast<long long>(g.nx) * g.ny;
    const int gx = g.nx / kCells;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= gx * g.ny) return;
    const int x0 = (t % gx) * kCells, y = t / gx;
    const int xy = y * g.nx + x0;
    for (int z = blockIdx.y; z < g.nz; z += gridDim.y) {
        const long long o = cell(g, x0, y, z);
        Real d[kCells], pp[kCells], ii[kCells], q[kCells], r[kCells], aq[kCells], ar[kCells];
        dval4(D, g, x0, y, z, d);
        ld4(P + o, pp);
        ld4(I + o, ii);
        ld4(Q + o, q);
        ld4(R + o, r);
        apply_A4(Q, d, g, x0, y, z, o, static_cast<const Real *>(nullptr), aq);
        apply_A4(R, d, g, x0, y, z, o, static_cast<const Real *>(nullptr), ar);
        const Real mk = Mk[z], mi = Mi[z];
        double gv[kCells];
        ld4(gV + o, gv);
#pragma unroll
        for (int k = 0; k < kCells; ++k) {
            Real pn, in;
            de_cell(g, pp[k], ii[k], q[k], r[k], mk, mi, aq[k], ar[k], gv[k], pn, in);
            if (kd >= 0) {
                if (z == kd) pn = fma(static_cast<Real>(w[xy + k]), Ist[plane + xy + k], pn);
                else if (z == kd + 1) pn = fma(-static_cast<Real>(w[xy + k]), Ist[xy + k], pn);
            }
            pp[k] = pn;
            ii[k] = in;
        }
        st4(gV + o, gv);
        st4(P + o, pp);
        st4(I + o, ii);
    }
}

// I^{-1/2} = Im psi0 - A R^0 / 2 makes L depend on V through the start: gV += (cv/2) Q R^0.
template <typename Real>
__global__ void adj_start_kernel(Geo g, const double *__restrict__ R0, const Real *__restrict__ Q,
                                 double *gV)
{
    const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
    GRID_STRIDE(t, n) gV[t] += 0.5 * g.cv * static_cast<double>(Q[t]) * R0[t];
}

template <typename Real>
__global__ void convert_kernel(long long n, const double *__restrict__ src, Real *dst)
{
    GRID_STRIDE(t, n) dst[t] = static_cast<Real>(src[t]);
}

// w = dL/dF * dt * cj per pixel
__global__ void flux_weight_kernel(long long npix, const double *__restrict__ gF, double scale,
                                   double *w)
{
    GRID_STRIDE(t, npix) w[t] = gF[t] * scale;
}

// ---------------------------------------------------------------- fused backward step
//
// Steps a-e above in one z-march per backward step.  A block owns a kTX x kTY tile of
// cells and a chunk [z0, z1) of planes, and keeps rings of planes in shared memory:
//   old I and P on the tile plus two cells (planes b-3 .. b+1),
//   old R and Q on the tile plus one cell (plane b), d on the tile plus one (b-2 .. b),
//   new R and Qt on the tile plus one cell (b-3 .. b).
// Iteration b: load I, P at plane b+1 and R, Q, d at plane b; step b at plane b on
// the tile plus one cell; the detector terms of step c once the new R of planes kd and
// kd+1 exist; steps d and e at plane q = b - 2 on the tile, written out.  Step b runs
// on planes [z0 - 2, z1 + 2), so the chunk's own rings hold every stencil operand of
// its planes (the one-cell ring of new R and Qt is recomputed by each tile that
// reads it), and every step reads one buffer set and writes the other: blocks never
// read what another block writes within a step.  Per cell and step it moves the
// fields once: R, I, P, Q, d and gV in, R, I, P, Q and gV out.
constexpr int kTX = 32, kTY = 8;                         // tile (one cell per thread)
constexpr int kW1 = kTX + 2, kH1 = kTY + 2, kA1 = kW1 * kH1;   // tile plus one cell
constexpr int kW2 = kTX + 4, kH2 = kTY + 4, kA2 = kW2 * kH2;   // tile plus two cells
constexpr int kRingIP = 5, kRingRQ = 4, kRingD = 3;

template <typename Real>
constexpr size_t fused_smem_bytes()
{
    return sizeof(Real) * (2 * kRingIP * kA2 + (2 + kRingD + 2 * kRingRQ) * kA1);
}

struct FusedArgs {
    Geo g;
    int kd;
    int tiles_x, tiles_y, chunk;
    const double *w;          // dL/dF dt cj per pixel
    const void *Mk, *Mi;      // absorbing factor per plane and its reciprocal
    const void *D;            // d of the forward step (padded)
    const void *R, *I, *P, *Q;     // state and adjoints read by this step
    void *Ro, *Io, *Po, *Qo;       // ... written by this step
    double *gV;
};

// A coordinate one of the grid's axes: the periodic image, or -1 beyond a wall.
__device__ __forceinline__ int wrap_axis(int v, int n, int per)
{
    if (v >= 0 && v < n) return v;
    if (!per) return -1;
    v %= n;
    return v < 0 ? v + n : v;
}

template <typename Real>
__device__ __forceinline__ Real plane_factor_any(const Real *__restrict__ sc, const Geo &g, int z)
{
    const int zz = wrap_axis(z, g.nz, g.per[2]);
    return zz < 0 ? Real(1) : sc[zz];
}

// Region of w x h cells at global (ox, oy) of plane z of an unpadded field into dst.
template <typename Real>
__device__ __forceinline__ void load_region(Real *__restrict__ dst, const Real *__restrict__ f,
                                            const Geo &g, int ox, int oy, int z, int w, int h)
{
    const int zz = wrap_axis(z, g.nz, g.per[2]);
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) {
        const int i = t % w, j = t / w;
        const int x = wrap_axis(ox + i, g.nx, g.per[0]), y = wrap_axis(oy + j, g.ny, g.per[1]);
        dst[t] = (zz < 0 || x < 0 || y < 0) ? Real(0) : f[cell(g, x, y, zz)];
    }
}

// The same for d, read from the forward step's padded array.
template <typename Real>
__device__ __forceinline__ void load_region_d(Real *__restrict__ dst, const Real *__restrict__ D,
                                              const Geo &g, int ox, int oy, int z, int w, int h)
{
    const int zz = wrap_axis(z, g.nz, g.per[2]);
    for (int t = threadIdx.x; t < w * h; t += blockDim.x) {
        const int i = t % w, j = t / w;
        const int x = wrap_axis(ox + i, g.nx, g.per[0]), y = wrap_axis(oy + j, g.ny, g.per[1]);
        dst[t] = (zz < 0 || x < 0 || y < 0)
                     ? Real(0)
                     : D[static_cast<long long>(zz) * g.pplane + static_cast<long long>(y + g.G) * g.pitch +
                         (x + g.G)];
    }
}

template <typename Real>
__global__ void __launch_bounds__(kTX * kTY) adj_fused_kernel(FusedArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    Real *sI = reinterpret_cast<Real *>(smem_raw);     // [kRingIP][kA2]
    Real *sP = sI + kRingIP * kA2;                     // [kRingIP][kA2]
    Real *sR = sP + kRingIP * kA2;                     // [kA1]
    Real *sQ = sR + kA1;                               // [kA1]
    Real *sD = sQ + kA1;                               // [kRingD][kA1]
    Real *sRn = sD + kRingD * kA1;                     // [kRingRQ][kA1]
    Real *sQt = sRn + kRingRQ * kA1;                   // [kRingRQ][kA1]

    const Geo &g = a.g;
    const int tiles = a.tiles_x * a.tiles_y;
    const int tile = blockIdx.x % tiles, chunk = blockIdx.x / tiles;
    const int x0 = (tile % a.tiles_x) * kTX, y0 = (tile / a.tiles_x) * kTY;
    const int z0 = chunk * a.chunk, z1 = min(z0 + a.chunk, g.nz);
    const Real *Mk = static_cast<const Real *>(a.Mk), *Mi = static_cast<const Real *>(a.Mi);
    const Real *D = static_cast<const Real *>(a.D);
    const Real *Rg = static_cast<const Real *>(a.R), *Ig = static_cast<const Real *>(a.I);
    const Real *Pg = static_cast<const Real *>(a.P), *Qg = static_cast<const Real *>(a.Q);
    const int kd = a.kd;
    auto ring = [](int z, int n) { return ((z % n) + n) % n; };

    // this thread's cell for steps d and e
    const int ti = threadIdx.x % kTX, tj = threadIdx.x / kTX;
    const int cx = x0 + ti, cy = y0 + tj;
    const bool own = cx < g.nx && cy < g.ny;
    const int c1 = (tj + 1) * kW1 + (ti + 1);     // its index in the one-cell regions
    const int c2 = (tj + 2) * kW2 + (ti + 2);     // ... and in the two-cell regions

    for (int z = z0 - 3; z <= z0 - 2; ++z) {      // the first planes of I and P
        load_region(sI + ring(z, kRingIP) * kA2, Ig, g, x0 - 2, y0 - 2, z, kW2, kH2);
        load_region(sP + ring(z, kRingIP) * kA2, Pg, g, x0 - 2, y0 - 2, z, kW2, kH2);
    }
    // The cells this thread loads in every plane (at most two of each region) as
    // offsets within a plane, -1 beyond a wall; the next plane's values are fetched
    // into registers while the current one is computed.
    constexpr int kN2 = (kA2 + kTX * kTY - 1) / (kTX * kTY), kN1 = (kA1 + kTX * kTY - 1) / (kTX * kTY);
    const long long plane = static_cast<long long>(g.nx) * g.ny;
    int xy2[kN2], xy1[kN1];
    long long dxy1[kN1];
#pragma unroll
    for (int k = 0; k < kN2; ++k) {
        const int t = threadIdx.x + k * kTX * kTY;
        const int x = wrap_axis(x0 - 2 + t % kW2, g.nx, g.per[0]), y = wrap_axis(y0 - 2 + t / kW2, g.ny, g.per[1]);
        xy2[k] = (t < kA2 && x >= 0 && y >= 0) ? y * g.nx + x : -1;
    }
#pragma unroll
    for (int k = 0; k < kN1; ++k) {
        const int t = threadIdx.x + k * kTX * kTY;
        const int x = wrap_axis(x0 - 1 + t % kW1, g.nx, g.per[0]), y = wrap_axis(y0 - 1 + t / kW1, g.ny, g.per[1]);
        const bool ok = t < kA1 && x >= 0 && y >= 0;
        xy1[k] = ok ? y * g.nx + x : -1;
        dxy1[k] = ok ? static_cast<long long>(y + g.G) * g.pitch + (x + g.G) : -1;
    }
    Real fI[kN2], fP[kN2], fR[kN1], fQ[kN1], fD[kN1];
    // I and P at plane zi, R, Q and d at plane zr into the fetch registers
    auto fetch = [&](int zi, int zr) {
        const int wi = wrap_axis(zi, g.nz, g.per[2]), wr = wrap_axis(zr, g.nz, g.per[2]);
#pragma unroll
        for (int k = 0; k < kN2; ++k) {
            const bool ok = wi >= 0 && xy2[k] >= 0;
            const long long o = wi * plane + xy2[k];
            fI[k] = ok ? Ig[o] : Real(0);
            fP[k] = ok ? Pg[o] : Real(0);
        }
#pragma unroll
        for (int k = 0; k < kN1; ++k) {
            const bool ok = wr >= 0 && xy1[k] >= 0;
            const long long o = wr * plane + xy1[k];
            fR[k] = ok ? Rg[o] : Real(0);
            fQ[k] = ok ? Qg[o] : Real(0);
            fD[k] = ok ? D[wr * g.pplane + dxy1[k]] : Real(0);
        }
    };
    auto deposit = [&](int zi, int zr) {
        Real *dI = sI + ring(zi, kRingIP) * kA2, *dP = sP + ring(zi, kRingIP) * kA2;
        Real *dD = sD + ring(zr, kRingD) * kA1;
#pragma unroll
        for (int k = 0; k < kN2; ++k) {
            const int t = threadIdx.x + k * kTX * kTY;
            if (t < kA2) {
                dI[t] = fI[k];
                dP[t] = fP[k];
            }
        }
#pragma unroll
        for (int k = 0; k < kN1; ++k) {
            const int t = threadIdx.x + k * kTX * kTY;
            if (t < kA1) {
                sR[t] = fR[k];
                sQ[t] = fQ[k];
                dD[t] = fD[k];
            }
        }
    };
    fetch(z0 - 1, z0 - 2);
    for (int b = z0 - 2; b <= z1 + 1; ++b) {
        __syncthreads();   // the previous iteration's reads of the slots refilled now are done
        deposit(b + 1, b);
        if (b + 1 <= z1 + 1) fetch(b + 2, b + 1);
        // dL/dV of the cell updated below (plane b - 2), fetched ahead of its use
        double gv = 0.0;
        const int qd = b - 2;
        const long long od = cell(g, min(cx, g.nx - 1), min(cy, g.ny - 1), max(qd, 0));
        if (qd >= z0 && qd < z1 && own) gv = a.gV[od];
        __syncthreads();
        // b. undo Eq. 8 and its adjoint at plane b on the tile plus one cell
        {
            const Real mi0 = plane_factor_any(Mi, g, b), mim = plane_factor_any(Mi, g, b - 1),
                       mip = plane_factor_any(Mi, g, b + 1);
            const Real mk0 = plane_factor_any(Mk, g, b), mkm = plane_factor_any(Mk, g, b - 1),
                       mkp = plane_factor_any(Mk, g, b + 1);
            const Real *I0 = sI + ring(b, kRingIP) * kA2, *Im = sI + ring(b - 1, kRingIP) * kA2,
                       *Ip = sI + ring(b + 1, kRingIP) * kA2;
            const Real *P0 = sP + ring(b, kRingIP) * kA2, *Pm = sP + ring(b - 1, kRingIP) * kA2,
                       *Pp = sP + ring(b + 1, kRingIP) * kA2;
            const Real *d0 = sD + ring(b, kRingD) * kA1;
            Real *Rn = sRn + ring(b, kRingRQ) * kA1, *Qt = sQt + ring(b, kRingRQ) * kA1;
            const bool zin = wrap_axis(b, g.nz, g.per[2]) >= 0;
            for (int t = threadIdx.x; t < kA1; t += blockDim.x) {
                const int i = t % kW1, j = t / kW1;
                const int k = (j + 1) * kW2 + (i + 1);     // same cell in the two-cell regions
                // beyond a wall the new R and Qt are zero, like every field there
                if (!zin || wrap_axis(x0 - 1 + i, g.nx, g.per[0]) < 0 || wrap_axis(y0 - 1 + j, g.ny, g.per[1]) < 0) {
                    Rn[t] = Real(0);
                    Qt[t] = Real(0);
                    continue;
                }
                const Real ai = stencil(g, rmul(I0[k - 1], mi0), rmul(I0[k + 1], mi0), rmul(I0[k - kW2], mi0),
                                        rmul(I0[k + kW2], mi0), rmul(Im[k], mim), rmul(Ip[k], mip),
                                        rmul(I0[k], mi0), d0[t]);
                const Real ap = stencil(g, rmul(P0[k - 1], mk0), rmul(P0[k + 1], mk0), rmul(P0[k - kW2], mk0),
                                        rmul(P0[k + kW2], mk0), rmul(Pm[k], mkm), rmul(Pp[k], mkp),
                                        rmul(P0[k], mk0), d0[t]);
                Rn[t] = fma(sR[t], mi0, ai);
                Qt[t] = fma(sQ[t], mk0, -ap);
            }
        }
        // c. the detector terms, once the new R of planes kd and kd + 1 exist (the
        // stencils of d and e below read only planes written before this iteration,
        // so only then is a barrier needed between the two)
        // (on a periodic z axis the chunk's planes may be images: compare the plane
        // itself, act on the ring slots of b - 1 and b)
        if (kd >= 0 && wrap_axis(b, g.nz, g.per[2]) == kd + 1 && b - 1 >= z0 - 2) {
            __syncthreads();
            Real *Qlo = sQt + ring(b - 1, kRingRQ) * kA1, *Qhi = sQt + ring(b, kRingRQ) * kA1;
            const Real *Rlo = sRn + ring(b - 1, kRingRQ) * kA1, *Rhi = sRn + ring(b, kRingRQ) * kA1;
            for (int t = threadIdx.x; t < kA1; t += blockDim.x) {
                const int x = wrap_axis(x0 - 1 + t % kW1, g.nx, g.per[0]);
                const int y = wrap_axis(y0 - 1 + t / kW1, g.ny, g.per[1]);
                if (x < 0 || y < 0) continue;
                const Real wp = static_cast<Real>(a.w[y * g.nx + x]);
                Qhi[t] = fma(wp, Rlo[t], Qhi[t]);
                Qlo[t] = fma(-wp, Rhi[t], Qlo[t]);
            }
            __syncthreads();
        }
        // d and e at plane q = b - 2 on the tile
        const int q = b - 2;
        if (q >= z0 && q < z1 && own) {
            const Real *Qq = sQt + ring(q, kRingRQ) * kA1, *Qm = sQt + ring(q - 1, kRingRQ) * kA1,
                       *Qp = sQt + ring(q + 1, kRingRQ) * kA1;
            const Real *Rq = sRn + ring(q, kRingRQ) * kA1, *Rm = sRn + ring(q - 1, kRingRQ) * kA1,
                       *Rp = sRn + ring(q + 1, kRingRQ) * kA1;
            const Real dq = sD[ring(q, kRingD) * kA1 + c1];
            const Real aq = stencil(g, Qq[c1 - 1], Qq[c1 + 1], Qq[c1 - kW1], Qq[c1 + kW1], Qm[c1], Qp[c1],
                                    Qq[c1], dq);
            const Real ar = stencil(g, Rq[c1 - 1], Rq[c1 + 1], Rq[c1 - kW1], Rq[c1 + kW1], Rm[c1], Rp[c1],
                                    Rq[c1], dq);
            const long long o = od;
            Real pn, in;
            de_cell(g, sP[ring(q, kRingIP) * kA2 + c2], sI[ring(q, kRingIP) * kA2 + c2], Qq[c1], Rq[c1],
                    Mk[q], Mi[q], aq, ar, gv, pn, in);
            if (kd >= 0 && (q == kd || q == kd + 1)) {
                const Real wp = static_cast<Real>(a.w[cy * g.nx + cx]);
                if (q == kd)   // It of plane kd + 1
                    pn = fma(wp, rmul(sI[ring(kd + 1, kRingIP) * kA2 + c2], Mi[kd + 1]), pn);
                else           // It of plane kd
                    pn = fma(-wp, rmul(sI[ring(kd, kRingIP) * kA2 + c2], Mi[kd]), pn);
            }
            a.gV[o] = gv;
            static_cast<Real *>(a.Ro)[o] = Rq[c1];
            static_cast<Real *>(a.Qo)[o] = Qq[c1];
            static_cast<Real *>(a.Po)[o] = pn;
            static_cast<Real *>(a.Io)[o] = in;
        }
    }
}

// ---------------------------------------------------------------- atom chain rule

// d phi / d(r^2) of the atom profile (see the potential kernel).
__device__ __forceinline__ void atom_profile(double r2, double a2, double rc, double *phi,
                                             double *dphi)
{
    const double rho = sqrt(r2 + a2);
    const double ir = 1.0 / rho, ir3 = ir * ir * ir;
    if (rc <= 0.0) {
        *phi = ir;
        *dphi = -0.5 * ir3;
        return;
    }
    const double uc = rc * rc;
    if (r2 >= uc) {
        *phi = 0.0;
        *dphi = 0.0;
        return;
    }
    const double ic = 1.0 / sqrt(uc + a2), ic3 = ic * ic * ic, ic5 = ic3 * ic * ic;
    const double du = r2 - uc;
    *phi = ir - (ic - 0.5 * du * ic3 + 0.375 * du * du * ic5);
    *dphi = -0.5 * ir3 - (-0.5 * ic3 + 0.75 * du * ic5);
}

struct AtomGeo {
    int nx, ny, nz;
    int per[3];
    double h[3], L[3];
    double a2, rc;
};

__device__ __forceinline__ double mimg(double d, double L, int per)
{
    return per ? d - L * floor(d / L + 0.5) : d;
}

// block (a, c): atom a, cells c, c + nchunk, ...; partial[(a * nchunk + c) * 4 + k]
__global__ void atom_grad_kernel(AtomGeo g, const double *__restrict__ atoms,
                                 const double *__restrict__ gV, int nchunk, double *partial)
{
    __shared__ double sh[4][kThreads / 32];
    const int a = blockIdx.x / nchunk, c = blockIdx.x % nchunk;
    const double ax = atoms[4 * a], ay = atoms[4 * a + 1], az = atoms[4 * a + 2], Z = atoms[4 * a + 3];
    const long long n = static_cast<long long>(g.nx) * g.ny * g.nz;
    double acc[4] = {0, 0, 0, 0};
    for (long long t = static_cast<long long>(c) * blockDim.x + threadIdx.x; t < n;
         t += static_cast<long long>(nchunk) * blockDim.x) {
        const int x = static_cast<int>(t % g.nx);
        const int y = static_cast<int>((t / g.nx) % g.ny);
        const int z = static_cast<int>(t / (static_cast<long long>(g.nx) * g.ny));
        const double dx = mimg(x * g.h[0] - ax, g.L[0], g.per[0]);
        const double dy = mimg(y * g.h[1] - ay, g.L[1], g.per[1]);
        const double dz = mimg(z * g.h[2] - az, g.L[2], g.per[2]);
        double phi, dphi;
        atom_profile(dx * dx + dy * dy + dz * dz, g.a2, g.rc, &phi, &dphi);
        const double wv = gV[t];
        // V_a = -Z phi(r^2), d(r^2)/d(x_a) = -2 (x - x_a)
        acc[0] += wv * 2.0 * Z * dphi * dx;
        acc[1] += wv * 2.0 * Z * dphi * dy;
        acc[2] += wv * 2.0 * Z * dphi * dz;
        acc[3] += wv * (-phi);
    }
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[k][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[threadIdx.x][w];
        partial[(static_cast<long long>(a) * nchunk + c) * 4 + threadIdx.x] = s;
    }
}

__global__ void atom_grad_finalize(int natoms, int nchunk, const double *__restrict__ partial,
                                   double *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= natoms * 4) return;
    const int a = i / 4, k = i % 4;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[(static_cast<long long>(a) * nchunk + c) * 4 + k];
    out[i] = s;
}

int grid_for(long long n)
{
    long long g = (n + kThreads - 1) / kThreads;
    if (g > 152LL * 64) g = 152LL * 64;
    return static_cast<int>(g < 1 ? 1 : g);
}

Geo make_geo(const MemberDev &m)
{
    Geo g;
    g.nx = m.nx;
    g.ny = m.ny;
    g.nz = m.nz;
    g.per[0] = m.per_x;
    g.per[1] = m.per_y;
    g.per[2] = m.per_z;
    g.cx = m.cx;
    g.cy = m.cy;
    g.cz = m.cz;
    g.cv = m.cv;
    g.c0 = -2.0 * (m.cx + m.cy + m.cz);
    g.pitch = m.pitch;
    g.pplane = m.plane;
    g.G = m.G;
    return g;
}

template <typename Real>
cudaError_t fused_step_t(const MemberDev &m, const AdjointBuffers &b, cudaStream_t s)
{
    FusedArgs a;
    a.g = make_geo(m);
    a.kd = m.det_k;
    a.tiles_x = (m.nx + kTX - 1) / kTX;
    a.tiles_y = (m.ny + kTY - 1) / kTY;
    // z-chunks: about four blocks per SM, at least 16 planes (each chunk recomputes
    // step b on four extra planes)
    const long long tiles = static_cast<long long>(a.tiles_x) * a.tiles_y;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long want = (4LL * sms + tiles - 1) / tiles;
    a.chunk = static_cast<int>(std::max<long long>(16, (m.nz + want - 1) / want));
    a.chunk = std::min(a.chunk, m.nz);
    const long long chunks = (m.nz + a.chunk - 1) / a.chunk;
    a.w = b.w;
    a.Mk = m.mask;
    a.Mi = b.Minv;
    a.D = m.d;
    a.R = b.R; a.I = b.I; a.P = b.P; a.Q = b.Q;
    a.Ro = b.R2; a.Io = b.I2; a.Po = b.P2; a.Qo = b.Q2;
    a.gV = b.gV;
    static std::atomic<uint64_t> smem_allowed{0};   // one bit per device
    const uint64_t bit = dev < 64 ? (uint64_t{1} << dev) : 0;
    if (!(bit && (smem_allowed.load() & bit))) {
        e = cudaFuncSetAttribute(adj_fused_kernel<Real>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(fused_smem_bytes<Real>()));
        if (e != cudaSuccess) return e;
        if (bit) smem_allowed.fetch_or(bit);
    }
    adj_fused_kernel<Real><<<static_cast<unsigned>(tiles * chunks), kTX * kTY, fused_smem_bytes<Real>(), s>>>(a);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t backward_step_t(const MemberDev &m, const AdjointBuffers &b, cudaStream_t s)
{
    if (b.R2) return fused_step_t<Real>(m, b, s);
    const Geo g = make_geo(m);
    const long long plane = static_cast<long long>(m.nx) * m.ny;
    // planes: one block row per plane up to 65535, then a plane-stride loop
    const dim3 grid(static_cast<unsigned>((plane / kCells + kThreads - 1) / kThreads),
                    static_cast<unsigned>(std::min(m.nz, 65535)));
    Real *R = static_cast<Real *>(b.R), *I = static_cast<Real *>(b.I);
    Real *P = static_cast<Real *>(b.P), *Q = static_cast<Real *>(b.Q);
    const Real *D = static_cast<const Real *>(m.d);
    const Real *Mk = static_cast<const Real *>(m.mask), *Mi = static_cast<const Real *>(b.Minv);
    Real *Ist = static_cast<Real *>(b.Ist);
    adj_b_kernel<Real><<<grid, kThreads, 0, s>>>(g, Mk, Mi, D, R, I, P, Q);
    const int kd = m.det_k;
    if (kd >= 0)
        adj_flux_q_kernel<Real><<<grid_for(plane), kThreads, 0, s>>>(g, kd, b.w, Mi, R, I, Q, Ist);
    adj_de_kernel<Real><<<grid, kThreads, 0, s>>>(g, Mk, Mi, D, kd, b.w, Ist, R, I, P, Q, b.gV);
    return cudaGetLastError();
}

}  // namespace

cudaError_t adjoint_backward_step(const MemberDev &m, int elem, const AdjointBuffers &b,
                                  cudaStream_t s)
{
    return elem == 8 ? backward_step_t<double>(m, b, s) : backward_step_t<float>(m, b, s);
}

cudaError_t adjoint_start_term(const MemberDev &m, int elem, const AdjointBuffers &b,
                               const double *R0, cudaStream_t s)
{
    const Geo g = make_geo(m);
    const long long n = static_cast<long long>(m.nx) * m.ny * m.nz;
    if (elem == 8)
        adj_start_kernel<double><<<grid_for(n), kThreads, 0, s>>>(g, R0, static_cast<double *>(b.Q), b.gV);
    else
        adj_start_kernel<float><<<grid_for(n), kThreads, 0, s>>>(g, R0, static_cast<float *>(b.Q), b.gV);
    return cudaGetLastError();
}

cudaError_t adjoint_load_state(const MemberDev &m, int elem, const AdjointBuffers &b,
                               const double *R64, const double *I64, cudaStream_t s)
{
    const long long n = static_cast<long long>(m.nx) * m.ny * m.nz;
    if (elem == 8) {
        cudaMemcpyAsync(b.R, R64, n * 8, cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(b.I, I64, n * 8, cudaMemcpyDeviceToDevice, s);
    } else {
        convert_kernel<float><<<grid_for(n), kThreads, 0, s>>>(n, R64, static_cast<float *>(b.R));
        convert_kernel<float><<<grid_for(n), kThreads, 0, s>>>(n, I64, static_cast<float *>(b.I));
    }
    return cudaGetLastError();
}

cudaError_t adjoint_flux_weights(const MemberDev &m, const double *gF, double *w, cudaStream_t s)
{
    const long long npix = static_cast<long long>(m.nx) * m.ny;
    flux_weight_kernel<<<grid_for(npix), kThreads, 0, s>>>(npix, gF, m.dt * m.cj, w);
    return cudaGetLastError();
}

int atom_grad_chunks() { return 256; }

cudaError_t launch_atom_gradient(const MemberDev &m, const double *atoms, int natoms, double a2,
                                 double rc, const double *gV, double *partial, double *out,
                                 cudaStream_t s)
{
    if (natoms <= 0) return cudaSuccess;
    AtomGeo g;
    g.nx = m.nx;
    g.ny = m.ny;
    g.nz = m.nz;
    g.per[0] = m.per_x;
    g.per[1] = m.per_y;
    g.per[2] = m.per_z;
    g.h[0] = m.hx;
    g.h[1] = m.hy;
    g.h[2] = m.hz;
    g.L[0] = m.nx * m.hx;
    g.L[1] = m.ny * m.hy;
    g.L[2] = m.nz * m.hz;
    g.a2 = a2;
    g.rc = rc;
    const int nchunk = atom_grad_chunks();
    atom_grad_kernel<<<natoms * nchunk, kThreads, 0, s>>>(g, atoms, gV, nchunk, partial);
    atom_grad_finalize<<<(natoms * 4 + 127) / 128, 128, 0, s>>>(natoms, nchunk, partial, out);
    return cudaGetLastError();
}

}  // namespace tdse
