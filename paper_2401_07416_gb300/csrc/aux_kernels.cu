// Set-up, conversion and reduction kernels of libtdse (everything except the
// fused step).  All arithmetic that feeds a reduction is FP64.
#include <algorithm>
#include <cmath>

#include "tdse_internal.cuh"

namespace tdse {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ long long pidx(const MemberDev &m, int x, int y, int z)
{
    return static_cast<long long>(z) * m.plane + static_cast<long long>(y + m.G) * m.pitch +
           (x + m.G);
}

__device__ __forceinline__ long long uidx(const MemberDev &m, int x, int y, int z)
{
    return (static_cast<long long>(z) * m.ny + y) * m.nx + x;
}

template <typename Real>
__device__ __forceinline__ double value(const MemberDev &m, const Real *f, const Real *c,
                                        long long o)
{
    double v = static_cast<double>(f[o]);
    if (c) v -= static_cast<double>(c[o]);
    return v;
}

// Visit every node: blocks take (y, z) rows through a 2-D grid, threads take x, so no
// index is split with a 64-bit division (a long software routine on the GPU).  f gets
// (x, y, z) and the unpadded linear index.
template <typename F>
__device__ __forceinline__ void for_each_node(int nx, int ny, int nz, F &&f)
{
    for (int z = blockIdx.y; z < nz; z += gridDim.y)
        for (int y = blockIdx.x; y < ny; y += gridDim.x) {
            const long long base = (static_cast<long long>(z) * ny + y) * nx;
            for (int x = threadIdx.x; x < nx; x += blockDim.x) f(x, y, z, base + x);
        }
}

// Field value at unpadded (x, y, z) with |x - x0|, |y - y0| <= 1 of an interior
// node: x/y come from the ghost zones, z wraps (periodic) or reads zero (wall).
template <typename Real>
__device__ __forceinline__ double nbr(const MemberDev &m, const Real *f, const Real *c, int x,
                                      int y, int z)
{
    if (z < 0 || z >= m.nz) {
        if (!m.per_z) return 0.0;
        z = (z % m.nz + m.nz) % m.nz;
    }
    return value<Real>(m, f, c, pidx(m, x, y, z));
}

// ---------------------------------------------------------------- ghost zones

// Ghost cells of each z plane (blocks take planes): the G rows below and above the
// interior (full padded width) and the G columns left and right of each interior row.
// A ghost takes the periodic image's interior value, or 0 beyond a wall.
template <typename Real>
__global__ void fill_ghosts_kernel(MemberDev m, Real *f)
{
    const int G = m.G, wx = m.nx + 2 * G;
    const int band = 2 * G * wx;                 // ghost rows of one plane
    const int ng = band + 2 * G * m.ny;          // + ghost columns
    for (int z = blockIdx.x; z < m.nz; z += gridDim.x)
        for (int e = threadIdx.x; e < ng; e += blockDim.x) {
            int x, y;
            if (e < band) {
                const int row = e / wx;          // 0 .. 2G-1
                x = e - row * wx - G;
                y = row < G ? row - G : m.ny + row - G;
            } else {
                const int c = e - band, row = c / (2 * G), k = c - row * 2 * G;
                y = row;
                x = k < G ? k - G : m.nx + k - G;
            }
            const bool gx = x < 0 || x >= m.nx, gy = y < 0 || y >= m.ny;
            Real v = Real(0);
            if ((!gx || m.per_x) && (!gy || m.per_y)) {
                const int sx = (x % m.nx + m.nx) % m.nx, sy = (y % m.ny + m.ny) % m.ny;
                v = f[pidx(m, sx, sy, z)];
            }
            f[pidx(m, x, y, z)] = v;
        }
}

// ---------------------------------------------------------------- potential

// One softened-Coulomb atom: phi(u = r^2) = f(u) - [f(uc) + f'(uc)(u - uc) +
// f''(uc)(u - uc)^2 / 2] for u < uc, f = (u + a^2)^-1/2, and 0 beyond.
__device__ __forceinline__ double atom_phi(double r2, double a2, double rc)
{
    const double rho = sqrt(r2 + a2);
    if (rc <= 0.0) return 1.0 / rho;
    const double uc = rc * rc;
    if (r2 >= uc) return 0.0;
    const double rhoc = sqrt(uc + a2);
    const double ic = 1.0 / rhoc, ic3 = ic * ic * ic, ic5 = ic3 * ic * ic;
    const double du = r2 - uc;
    return 1.0 / rho - (ic - 0.5 * du * ic3 + 0.375 * du * du * ic5);
}

// Atom position in grid units: node index i0 and fraction f in [0, 1), so that
// the distance to node i along the axis is h (i - i0 - f) with the integer part
// exact (and the periodic minimum image an integer wrap).
struct AtomCell {
    int i[3];
    float f[3];
    double fd[3];
    double Z;
};

__global__ void atom_cells_kernel(MemberDev m, const double *__restrict__ atoms, int n,
                                  AtomCell *__restrict__ out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    const double h[3] = {m.hx, m.hy, m.hz};
    AtomCell c;
    for (int k = 0; k < 3; ++k) {
        const double u = atoms[4 * a + k] / h[k];
        const double fl = floor(u);
        c.i[k] = static_cast<int>(fl);
        c.fd[k] = u - fl;
        c.f[k] = static_cast<float>(c.fd[k]);
    }
    c.Z = atoms[4 * a + 3];
    out[a] = c;
}

// Integer offset i - i0 along an axis of n nodes, wrapped to the nearest periodic
// image ([-n/2, n/2]) on a periodic axis.
__device__ __forceinline__ int wrap_offset(int k, int n, int periodic)
{
    if (periodic) {
        k %= n;
        if (k > n / 2) k -= n;
        if (k < -n / 2) k += n;
    }
    return k;
}

// V at every node from the atoms.  FP64 contexts evaluate each term in FP64;
// FP32 contexts evaluate the profile in FP32 (V is stored in FP32 for the step)
// from exact integer offsets, accumulating with compensated FP32 additions.
template <typename Compute>
__global__ void potential_kernel(MemberDev m, const AtomCell *__restrict__ atoms, int n,
                                 double a2, double rc, double *__restrict__ V)
{
    __shared__ AtomCell sa[128];
    const long long cells = static_cast<long long>(m.nx) * m.ny * m.nz;
    const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    const int x = static_cast<int>(t % m.nx);
    const int y = static_cast<int>((t / m.nx) % m.ny);
    const int z = static_cast<int>(t / (static_cast<long long>(m.nx) * m.ny));
    const Compute h[3] = {static_cast<Compute>(m.hx), static_cast<Compute>(m.hy),
                          static_cast<Compute>(m.hz)};
    const Compute ca2 = static_cast<Compute>(a2);
    // profile phi(u) = (u + a^2)^-1/2 - [p0 + p1 (u - uc) + p2 (u - uc)^2] for u < uc
    const double uc = rc > 0.0 ? rc * rc : 0.0;
    const double ic = rc > 0.0 ? 1.0 / sqrt(uc + a2) : 0.0;
    const Compute p0 = static_cast<Compute>(ic), p1 = static_cast<Compute>(-0.5 * ic * ic * ic),
                  p2 = static_cast<Compute>(0.375 * ic * ic * ic * ic * ic);
    const Compute cuc = static_cast<Compute>(uc);
    const bool cut = rc > 0.0;
    Compute acc = Compute(0), comp = Compute(0);
    for (int a0 = 0; a0 < n; a0 += 128) {
        const int na = min(128, n - a0);
        __syncthreads();
        if (threadIdx.x < na) sa[threadIdx.x] = atoms[a0 + threadIdx.x];
        __syncthreads();
        if (t >= cells) continue;
        for (int a = 0; a < na; ++a) {
            const AtomCell &c = sa[a];
            const int kx = wrap_offset(x - c.i[0], m.nx, m.per_x);
            const int ky = wrap_offset(y - c.i[1], m.ny, m.per_y);
            const int kz = wrap_offset(z - c.i[2], m.nz, m.per_z);
            Compute gx, gy, gz;   // offsets in grid units, nearest image on periodic axes
            if constexpr (sizeof(Compute) == 8) {
                gx = kx - c.fd[0];
                gy = ky - c.fd[1];
                gz = kz - c.fd[2];
            } else {
                gx = static_cast<float>(kx) - c.f[0];
                gy = static_cast<float>(ky) - c.f[1];
                gz = static_cast<float>(kz) - c.f[2];
            }
            if (m.per_x && gx < Compute(-0.5) * m.nx) gx += m.nx;
            if (m.per_y && gy < Compute(-0.5) * m.ny) gy += m.ny;
            if (m.per_z && gz < Compute(-0.5) * m.nz) gz += m.nz;
            const Compute dx = h[0] * gx, dy = h[1] * gy, dz = h[2] * gz;
            const Compute u = fma(dx, dx, fma(dy, dy, dz * dz));
            if (cut && u >= cuc) continue;   // beyond the cut-off the profile is zero
            Compute phi;
            if constexpr (sizeof(Compute) == 8) {
                phi = rsqrt(u + ca2);   // library reciprocal square root (within 1 ulp)
            } else {
                phi = rsqrtf(u + ca2);
            }
            if (cut) {
                const Compute du = u - cuc;
                phi -= fma(fma(p2, du, p1), du, p0);
            }
            const Compute term = -static_cast<Compute>(c.Z) * phi;
            if constexpr (sizeof(Compute) == 8) {
                acc += term;
            } else {
                const Compute yk = term - comp;
                const Compute tk = acc + yk;
                comp = (tk - acc) - yk;
                acc = tk;
            }
        }
    }
    if (t < cells) V[t] = static_cast<double>(acc) - static_cast<double>(comp);
}

// d = -2 (cx + cy + cz) - cv V into the padded Real array; V kept in FP64 (V may be
// V64 itself: the potential was written there directly).
template <typename Real>
__global__ void build_d_kernel(MemberDev m, const double *V, Real *d, double *V64)
{
    const double c0 = -2.0 * (m.cx + m.cy + m.cz);
    for_each_node(m.nx, m.ny, m.nz, [&](int x, int y, int z, long long t) {
        const double v = V ? V[t] : 0.0;
        if (V != V64) V64[t] = v;
        d[pidx(m, x, y, z)] = static_cast<Real>(c0 - m.cv * v);
    });
}

// ---------------------------------------------------------------- wave packet

struct PacketArgs {
    double r0[3], sigma[3], k0[3];
};

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (blockDim.x + 31) / 32; ++w) s += sh[w];
    return s;   // valid in thread 0
}

// Eq. 3 factorises over the axes: psi0(r) = prod_a g_a(r_a) exp(i k_a (r_a - r0_a)) with
// g_a = exp(-(r_a - r0_a)^2 / (2 sigma_a^2)) (1 on a plane-wave axis, sigma_a <= 0).
// So does the kinetic part of A psi0 (Eq. 7): the second difference along axis a acts
// on that axis' factor alone, c_a (f_a(i+1) + f_a(i-1)) times the other two factors,
// with the neighbour wrapped on a periodic axis and zero beyond a wall.
// One block per axis writes the axis' complex factors f_a, its neighbour sums
// c_a (f_a(i+1) + f_a(i-1)) and the sum of |f_a|^2; the product of the three sums
// times h^3 is the discrete norm of psi0.
__global__ void packet_axes_kernel(MemberDev m, PacketArgs P, double2 *__restrict__ fac,
                                   double2 *__restrict__ nsum, double *__restrict__ sums)
{
    __shared__ double sh[32];
    const int a = blockIdx.x;
    const int n = a == 0 ? m.nx : a == 1 ? m.ny : m.nz;
    const double h = a == 0 ? m.hx : a == 1 ? m.hy : m.hz;
    const double c = a == 0 ? m.cx : a == 1 ? m.cy : m.cz;
    const bool per = a == 0 ? m.per_x : a == 1 ? m.per_y : m.per_z;
    const int off = a == 0 ? 0 : a == 1 ? m.nx : m.nx + m.ny;
    double2 *f = fac + off;
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double d = i * h - P.r0[a];
        const double amp = P.sigma[a] > 0.0 ? exp(-d * d / (2.0 * P.sigma[a] * P.sigma[a])) : 1.0;
        double sn, cs;
        sincos(P.k0[a] * d, &sn, &cs);
        f[i] = make_double2(amp * cs, amp * sn);
        acc += amp * amp;
    }
    const double s = block_sum(acc, sh);   // its barriers order the f[] writes before the reads below
    if (threadIdx.x == 0) sums[a] = s;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double2 lo = make_double2(0.0, 0.0), hi = make_double2(0.0, 0.0);
        if (i > 0) lo = f[i - 1];
        else if (per) lo = f[n - 1];
        if (i + 1 < n) hi = f[i + 1];
        else if (per) hi = f[0];
        nsum[off + i] = make_double2(c * (lo.x + hi.x), c * (lo.y + hi.y));
    }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Row factors of the packet: for every (y, z) row, gh = f_y f_z and
// u = n_y f_z + f_y n_z (n: the neighbour sums above), so that at (x, y, z)
//   psi0 = f_x gh   and   kinetic part of A psi0 = n_x gh + f_x u.
__global__ void packet_rows_kernel(MemberDev m, const double2 *__restrict__ fac,
                                   const double2 *__restrict__ nsum, double2 *__restrict__ rows)
{
    for (int z = blockIdx.x; z < m.nz; z += gridDim.x)
        for (int y = threadIdx.x; y < m.ny; y += blockDim.x) {
        const long long r = static_cast<long long>(z) * m.ny + y;
        const double2 fy = fac[m.nx + y], fz = fac[m.nx + m.ny + z];
        const double2 ny = nsum[m.nx + y], nz = nsum[m.nx + m.ny + z];
        const double2 a = cmul(ny, fz), b = cmul(fy, nz);
        rows[2 * r] = cmul(fy, fz);
        rows[2 * r + 1] = make_double2(a.x + b.x, a.y + b.y);
    }
}

// R^0 = s Re psi0 and I^{-1/2} = s (Im psi0 - A[Re psi0] / 2) (Sec. 2.1), stored as
// Real (+ the compensation terms), s = 1 / sqrt(h^3 Sx Sy Sz).  A is real, so
// A[Re psi0] = Re(kinetic part of A psi0) + (d - cv V) Re psi0 with d = -2 (cx+cy+cz).
template <typename Real>
__global__ void packet_start_kernel(MemberDev m, const double *__restrict__ V64,
                                    const double2 *__restrict__ fac, const double2 *__restrict__ nsum,
                                    const double2 *__restrict__ rows, const double *__restrict__ sums,
                                    int kahan, int buf)
{
    const double s = 1.0 / sqrt(m.hx * m.hy * m.hz * sums[0] * sums[1] * sums[2]);
    Real *oR = reinterpret_cast<Real *>(m.R[buf]);
    Real *oI = reinterpret_cast<Real *>(m.I[buf]);
    Real *oCR = reinterpret_cast<Real *>(m.cR[buf]);
    Real *oCI = reinterpret_cast<Real *>(m.cI[buf]);
    const double c0 = -2.0 * (m.cx + m.cy + m.cz);
    for_each_node(m.nx, m.ny, m.nz, [&](int x, int y, int z, long long t) {
        const long long r = static_cast<long long>(z) * m.ny + y;
        const double2 f = fac[x], n = nsum[x], gh = rows[2 * r], u = rows[2 * r + 1];
        const double re = f.x * gh.x - f.y * gh.y;
        const double im = f.x * gh.y + f.y * gh.x;
        const double kin = (n.x * gh.x - n.y * gh.y) + (f.x * u.x - f.y * u.y);
        const double ar = kin + (c0 - m.cv * V64[t]) * re;
        const double rv = s * re;
        const double iv = s * (im - 0.5 * ar);
        const long long o = pidx(m, x, y, z);
        const Real rs = static_cast<Real>(rv), is = static_cast<Real>(iv);
        oR[o] = rs;
        oI[o] = is;
        if (kahan) {
            oCR[o] = static_cast<Real>(static_cast<double>(rs) - rv);
            oCI[o] = static_cast<Real>(static_cast<double>(is) - iv);
        }
    });
}

// ---------------------------------------------------------------- state copies

template <typename Real>
__global__ void set_state_kernel(MemberDev m, const double *__restrict__ R,
                                 const double *__restrict__ I, int kahan, int buf)
{
    Real *oR = reinterpret_cast<Real *>(m.R[buf]);
    Real *oI = reinterpret_cast<Real *>(m.I[buf]);
    Real *oCR = reinterpret_cast<Real *>(m.cR[buf]);
    Real *oCI = reinterpret_cast<Real *>(m.cI[buf]);
    for_each_node(m.nx, m.ny, m.nz, [&](int x, int y, int z, long long t) {
        const long long o = pidx(m, x, y, z);
        const Real rs = static_cast<Real>(R[t]), is = static_cast<Real>(I[t]);
        oR[o] = rs;
        oI[o] = is;
        if (kahan) {
            oCR[o] = static_cast<Real>(static_cast<double>(rs) - R[t]);
            oCI[o] = static_cast<Real>(static_cast<double>(is) - I[t]);
        }
    });
}

template <typename Real>
__global__ void get_state_kernel(MemberDev m, double *__restrict__ R, double *__restrict__ I,
                                 int kahan, int buf)
{
    const Real *iR = reinterpret_cast<const Real *>(m.R[buf]);
    const Real *iI = reinterpret_cast<const Real *>(m.I[buf]);
    const Real *iCR = kahan ? reinterpret_cast<const Real *>(m.cR[buf]) : nullptr;
    const Real *iCI = kahan ? reinterpret_cast<const Real *>(m.cI[buf]) : nullptr;
    for_each_node(m.nx, m.ny, m.nz, [&](int x, int y, int z, long long t) {
        const long long o = pidx(m, x, y, z);
        if (R) R[t] = value<Real>(m, iR, iCR, o);
        if (I) I[t] = value<Real>(m, iI, iCI, o);
    });
}

// Interior of a padded Real field <-> unpadded FP64 array (exact in both directions
// for values that are Real).
template <typename Real>
__global__ void field_io_kernel(MemberDev m, Real *field, double *host_side, int to_field)
{
    for_each_node(m.nx, m.ny, m.nz, [&](int x, int y, int z, long long t) {
        const long long o = pidx(m, x, y, z);
        if (to_field)
            field[o] = static_cast<Real>(host_side[t]);
        else
            host_side[t] = static_cast<double>(field[o]);
    });
}

// ---------------------------------------------------------------- observables

// Per block: sums of (R.R + I+.I, R^2 + I^2, R.AR + I+.AI) with I+ = I + A R.
// One thread per (x, y) column marching along z with a register window of R and
// I at z-1, z, z+1; x/y neighbours come from the ghost zones.  FP64 contexts do
// everything in FP64.  FP32 contexts evaluate the stencil and the per-node
// products in FP32 (the arithmetic of the step itself; Kahan compensation terms
// are below that resolution) and sum each column with compensated FP32
// additions before adding it to the FP64 accumulators.
template <typename Real>
struct ColumnSum {
    Real s = Real(0), c = Real(0);
    __device__ __forceinline__ void add(Real x)
    {
        const Real y = x - c;
        const Real t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const
    {
        return static_cast<double>(s) - static_cast<double>(c);
    }
};

// FP64 contexts: the column sums are plain FP64 additions.
template <>
struct ColumnSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};

// Sums of the detector flux map (last step and time-integrated) over block lb's
// share (of nb) of the pixels.
__device__ __forceinline__ void flux_partials(const MemberDev &m, double &fl, double &fi, int lb, int nb)
{
    if (m.det_k < 0) return;
    const long long npix = static_cast<long long>(m.nx) * m.ny;
    for (long long i = lb * static_cast<long long>(blockDim.x) + threadIdx.x; i < npix;
         i += static_cast<long long>(nb) * blockDim.x) {
        fl += m.jlast[i];
        fi += m.flux[i];
    }
}

__device__ __forceinline__ void write_partials(double *partials, double *sh, double q, double pn,
                                               double e, double fl, double fi, int lb)
{
    const double v[5] = {q, pn, e, fl, fi};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double t = block_sum(v[k], sh);
        if (threadIdx.x == 0) partials[kObsPartialsPerBlock * lb + k] = t;
    }
}

// Q, paper norm and energy numerator over (column group, z-chunk) items: each
// thread marches a chunk of zch planes of V adjacent (x, y) columns (one 16-byte
// vector per field and plane) with a three-plane window and accumulates the chunk
// in ColumnSum.  Items go to threads in a fixed order and the block count is fixed
// by the grid shape, so the sums are reproducible.  V = 1 is the scalar form for
// rows whose length is not a multiple of the vector width.
// Block lb of the nb blocks that reduce member m (the work of one block of
// observables_kernel, wherever it is launched).
template <typename Real, int V, int ZC>
__device__ __forceinline__ void observables_block(const MemberDev &m, int buf, double *__restrict__ partials,
                                                  int zch_arg, int lb, int nb, double *sh)
{
    const int zch = ZC > 0 ? ZC : zch_arg;   // ZC > 0: the chunk is a compile-time constant
    const Real *__restrict__ R = reinterpret_cast<const Real *>(m.R[buf]);
    const Real *__restrict__ I = reinterpret_cast<const Real *>(m.I[buf]);
    const Real *__restrict__ D = reinterpret_cast<const Real *>(m.d);
    const int ngx = m.nx / V;
    const int ngrp = ngx * m.ny;             // < 2^31: nx * ny is at most a few million
    const int nch = (m.nz + zch - 1) / zch;
    const long long nitems = static_cast<long long>(ngrp) * nch;
    const Real cx = static_cast<Real>(m.cx), cy = static_cast<Real>(m.cy),
               cz = static_cast<Real>(m.cz);
    const long long plane = m.plane;
    const int pitch = static_cast<int>(m.pitch);
    auto ld = [](const Real *p, Real (&v)[V]) {
        if constexpr (V * sizeof(Real) == 16) {
            if constexpr (sizeof(Real) == 4) {
                const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
                v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
            } else {
                const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
                v[0] = t.x; v[1] = t.y;
            }
        } else if constexpr (V == 2 && sizeof(Real) == 4) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
            v[0] = t.x; v[1] = t.y;
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) v[k] = __ldg(p + k);
        }
    };
    double q = 0.0, pn = 0.0, e = 0.0;
    for (long long item = lb * static_cast<long long>(blockDim.x) + threadIdx.x;
         item < nitems; item += static_cast<long long>(nb) * blockDim.x) {
        const int ch = static_cast<int>(item / ngrp);
        const int grp = static_cast<int>(item - static_cast<long long>(ch) * ngrp);
        const int z0 = ch * zch;
        const int z1 = min(z0 + zch, m.nz);
        const int x0 = (grp % ngx) * V, y = grp / ngx;
        const long long base = static_cast<long long>(y + m.G) * pitch + (x0 + m.G);
        // running pointers to this column's node at plane z (advanced by one plane)
        const Real *pr = R + base + static_cast<long long>(z0) * plane;
        const Real *pi = I + base + static_cast<long long>(z0) * plane;
        const Real *pd = D + base + static_cast<long long>(z0) * plane;
        Real rm[V], rc[V], im[V], ic[V];
        if (z0 > 0) {
            ld(pr - plane, rm);
            ld(pi - plane, im);
        } else if (m.per_z) {
            ld(pr + static_cast<long long>(m.nz - 1) * plane, rm);
            ld(pi + static_cast<long long>(m.nz - 1) * plane, im);
        } else {
#pragma unroll
            for (int k = 0; k < V; ++k) rm[k] = im[k] = Real(0);
        }
        ld(pr, rc);
        ld(pi, ic);
        ColumnSum<Real> sq, sp, se;
        // the plane at pr / pi / pd, its z+1 neighbours given
        auto plane_terms = [&](const Real (&rp)[V], const Real (&ip)[V]) {
            Real d[V], ryp[V], rym[V], iyp[V], iym[V];
            ld(pd, d);
            ld(pr + pitch, ryp);
            ld(pr - pitch, rym);
            ld(pi + pitch, iyp);
            ld(pi - pitch, iym);
            const Real rxl = __ldg(pr - 1), rxr = __ldg(pr + V);
            const Real ixl = __ldg(pi - 1), ixr = __ldg(pi + V);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                const Real rsx = (k == 0 ? rxl : rc[k - 1]) + (k == V - 1 ? rxr : rc[k + 1]);
                const Real isx = (k == 0 ? ixl : ic[k - 1]) + (k == V - 1 ? ixr : ic[k + 1]);
                const Real ar = fma(cx, rsx, fma(cy, ryp[k] + rym[k], fma(cz, rm[k] + rp[k], d[k] * rc[k])));
                const Real ai = fma(cx, isx, fma(cy, iyp[k] + iym[k], fma(cz, im[k] + ip[k], d[k] * ic[k])));
                const Real ipl = ic[k] + ar;
                sq.add(rc[k] * rc[k] + ipl * ic[k]);
                sp.add(rc[k] * rc[k] + ic[k] * ic[k]);
                se.add(rc[k] * ar + ipl * ai);
            }
#pragma unroll
            for (int k = 0; k < V; ++k) {
                rm[k] = rc[k];
                rc[k] = rp[k];
                im[k] = ic[k];
                ic[k] = ip[k];
            }
        };
        const int zin = min(z1, m.nz - 1);   // planes whose z+1 neighbour lies in the grid
#pragma unroll 2
        for (int z = z0; z < zin; ++z) {
            Real rp[V], ip[V];
            ld(pr + plane, rp);
            ld(pi + plane, ip);
            plane_terms(rp, ip);
            pr += plane;
            pi += plane;
            pd += plane;
        }
        if (z1 == m.nz) {   // top plane: periodic wrap or wall
            Real rp[V], ip[V];
            if (m.per_z) {
                ld(R + base, rp);
                ld(I + base, ip);
            } else {
#pragma unroll
                for (int k = 0; k < V; ++k) rp[k] = ip[k] = Real(0);
            }
            plane_terms(rp, ip);
        }
        q += sq.value();
        pn += sp.value();
        e += se.value();
    }
    double fl = 0.0, fi = 0.0;
    flux_partials(m, fl, fi, lb, nb);
    write_partials(partials, sh, q, pn, e, fl, fi, lb);
}

template <typename Real, int V, int ZC>
__global__ void __launch_bounds__(kObsThreads, kObsBlocksPerSM)
    observables_kernel(MemberDev m, int buf, double *__restrict__ partials, int zch_arg)
{
    __shared__ double sh[32];
    observables_block<Real, V, ZC>(m, buf, partials, zch_arg, blockIdx.x, gridDim.x, sh);
}

// Every member of a batch in one launch: block b belongs to the member whose slice
// of blocks contains it and does exactly the work of that member's block b - begin
// in a launch of its own (same items, same order), so the sums are the same bits.
template <typename Real, int V>
__global__ void __launch_bounds__(kObsThreads, kObsBlocksPerSM)
    observables_batch_kernel(const MemberDev *__restrict__ members, const ObsSlice *__restrict__ slices,
                             int nmembers, int buf, double *__restrict__ partials)
{
    __shared__ double sh[32];
    int mm = 0;
    while (mm + 1 < nmembers && static_cast<int>(blockIdx.x) >= slices[mm + 1].block_begin) ++mm;
    const ObsSlice sl = slices[mm];
    observables_block<Real, V, 0>(members[mm], buf, partials + kObsPartialsPerBlock * sl.block_begin, sl.zch,
                                  static_cast<int>(blockIdx.x) - sl.block_begin, sl.nparts, sh);
}

// record = {step, Q, norm_paper, energy, flux_last, flux_integrated}; sets
// status bit 1 on non-finite Q or Q > (1 + 1e-3) q_ref (q_ref <= 0: no check).
__device__ __forceinline__ void observables_finalize_block(const MemberDev &m, const double *__restrict__ partials,
                                                           int nparts, double *__restrict__ record,
                                                           int *status, double q_ref, long long step,
                                                           double *sh)
{
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nparts; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) v[k] += partials[kObsPartialsPerBlock * i + k];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = block_sum(v[k], sh);
    if (threadIdx.x == 0) {
        const double q = v[0], pn = v[1], e = v[2], fl = v[3], fi = v[4];
        const double h3 = m.hx * m.hy * m.hz;
        const double hxy = m.hx * m.hy;
        record[0] = static_cast<double>(step);
        record[1] = q * h3;
        record[2] = pn * h3;
        record[3] = -(m.hbar / m.dt) * e / q;
        record[4] = fl * hxy;
        record[5] = fi * hxy;
        if (!isfinite(q * h3) || !isfinite(e) || (q_ref > 0.0 && q * h3 > q_ref * (1.0 + 1e-3)))
            atomicOr(status, 2);
    }
}

__global__ void observables_finalize_kernel(MemberDev m, const double *__restrict__ partials,
                                            int nparts, double *__restrict__ record,
                                            int *status, double q_ref, long long step)
{
    __shared__ double sh[32];
    observables_finalize_block(m, partials, nparts, record, status, q_ref, step, sh);
}

// One block per member of a batch: its record goes to records + member * rec_stride.
__global__ void observables_batch_finalize_kernel(const MemberDev *__restrict__ members,
                                                  const ObsSlice *__restrict__ slices,
                                                  const double *__restrict__ partials,
                                                  double *__restrict__ records, long long rec_stride,
                                                  int *status, long long step)
{
    __shared__ double sh[32];
    const ObsSlice sl = slices[blockIdx.x];
    observables_finalize_block(members[blockIdx.x], partials + kObsPartialsPerBlock * sl.block_begin,
                               sl.nparts, records + blockIdx.x * rec_stride, status, sl.q_ref, step, sh);
}

int grid_for(long long n)
{
    long long g = (n + kThreads - 1) / kThreads;
    if (g > 65535LL * 32) g = 65535LL * 32;
    if (g < 1) g = 1;
    return static_cast<int>(g);
}

// Launch shape of a for_each_node kernel: a warp multiple of threads up to kThreads
// along x, and about two waves of blocks over the (y, z) rows.
struct NodeLaunch {
    dim3 grid;
    int threads;
};

NodeLaunch node_launch(int nx, int ny, int nz)
{
    const int threads = nx >= kThreads ? kThreads : std::max(32, (nx + 31) / 32 * 32);
    const int target = 2 * 152 * (2048 / threads);
    const int gx = std::min(ny, 64);
    const int gy = std::max(1, std::min({nz, 65535, std::max(1, target / gx)}));
    return {dim3(static_cast<unsigned>(gx), static_cast<unsigned>(gy)), threads};
}

NodeLaunch node_launch(const MemberDev &m) { return node_launch(m.nx, m.ny, m.nz); }

}  // namespace

cudaError_t launch_fill_ghosts(const MemberDev &m, void *field, int elem, cudaStream_t s)
{
    const int planes = std::min(m.nz, 152 * 16);
    if (elem == 8)
        fill_ghosts_kernel<double><<<planes, kThreads, 0, s>>>(m, static_cast<double *>(field));
    else
        fill_ghosts_kernel<float><<<planes, kThreads, 0, s>>>(m, static_cast<float *>(field));
    return cudaGetLastError();
}

cudaError_t launch_potential_atoms(const MemberDev &m, const double *atoms, int n, double a2,
                                   double rc, double *V, void *scratch, int precision,
                                   cudaStream_t s)
{
    const long long cells = static_cast<long long>(m.nx) * m.ny * m.nz;
    AtomCell *ac = static_cast<AtomCell *>(scratch);
    if (n > 0) atom_cells_kernel<<<(n + 127) / 128, 128, 0, s>>>(m, atoms, n, ac);
    const unsigned blocks = static_cast<unsigned>((cells + 127) / 128);
    if (precision == 0)
        potential_kernel<double><<<blocks, 128, 0, s>>>(m, ac, n, a2, rc, V);
    else
        potential_kernel<float><<<blocks, 128, 0, s>>>(m, ac, n, a2, rc, V);
    return cudaGetLastError();
}

size_t atom_cell_bytes(int n) { return static_cast<size_t>(n > 0 ? n : 1) * sizeof(AtomCell); }

cudaError_t launch_build_d(const MemberDev &m, int elem, const double *V, double *V64,
                           cudaStream_t s)
{
    const NodeLaunch L = node_launch(m);
    if (elem == 8)
        build_d_kernel<double><<<L.grid, L.threads, 0, s>>>(m, V, static_cast<double *>(m.d), V64);
    else
        build_d_kernel<float><<<L.grid, L.threads, 0, s>>>(m, V, static_cast<float *>(m.d), V64);
    return cudaGetLastError();
}

size_t packet_scratch_bytes(const MemberDev &m)
{
    const size_t axes = static_cast<size_t>(m.nx) + m.ny + m.nz;
    const size_t rows = static_cast<size_t>(m.ny) * m.nz;
    return (2 * axes + 2 * rows) * sizeof(double2) + 4 * sizeof(double);
}

cudaError_t launch_packet_start(const MemberDev &m, const double *V64, const double *r0,
                                const double *sigma, const double *k0, void *scratch,
                                int precision, int buf, cudaStream_t s)
{
    PacketArgs P;
    for (int a = 0; a < 3; ++a) {
        P.r0[a] = r0[a];
        P.sigma[a] = sigma[a];
        P.k0[a] = k0[a];
    }
    const size_t axes = static_cast<size_t>(m.nx) + m.ny + m.nz;
    const long long nrows = static_cast<long long>(m.ny) * m.nz;
    const NodeLaunch L = node_launch(m);
    double2 *fac = static_cast<double2 *>(scratch);
    double2 *nsum = fac + axes;
    double2 *rows = nsum + axes;
    double *sums = reinterpret_cast<double *>(rows + 2 * nrows);
    packet_axes_kernel<<<3, kThreads, 0, s>>>(m, P, fac, nsum, sums);
    packet_rows_kernel<<<std::min(m.nz, 152 * 16), kThreads, 0, s>>>(m, fac, nsum, rows);
    if (precision == 0)
        packet_start_kernel<double><<<L.grid, L.threads, 0, s>>>(m, V64, fac, nsum, rows, sums, 0, buf);
    else
        packet_start_kernel<float><<<L.grid, L.threads, 0, s>>>(m, V64, fac, nsum, rows, sums,
                                                                precision == 2, buf);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const MemberDev &m, const double *R64, const double *I64,
                             int precision, int buf, cudaStream_t s)
{
    const NodeLaunch L = node_launch(m);
    if (precision == 0)
        set_state_kernel<double><<<L.grid, L.threads, 0, s>>>(m, R64, I64, 0, buf);
    else
        set_state_kernel<float><<<L.grid, L.threads, 0, s>>>(m, R64, I64, precision == 2, buf);
    return cudaGetLastError();
}

cudaError_t launch_get_state(const MemberDev &m, double *R64, double *I64, int precision,
                             int buf, cudaStream_t s)
{
    const NodeLaunch L = node_launch(m);
    if (precision == 0)
        get_state_kernel<double><<<L.grid, L.threads, 0, s>>>(m, R64, I64, 0, buf);
    else
        get_state_kernel<float><<<L.grid, L.threads, 0, s>>>(m, R64, I64, precision == 2, buf);
    return cudaGetLastError();
}

cudaError_t launch_field_io(const MemberDev &m, void *field, int elem, double *array, int to_field,
                            cudaStream_t s)
{
    const NodeLaunch L = node_launch(m);
    if (elem == 8)
        field_io_kernel<double><<<L.grid, L.threads, 0, s>>>(m, static_cast<double *>(field), array, to_field);
    else
        field_io_kernel<float><<<L.grid, L.threads, 0, s>>>(m, static_cast<float *>(field), array, to_field);
    return cudaGetLastError();
}

// Trilinear interpolation of a periodic cell lattice Vc[cnz][cny][cnx] (cell lengths L,
// lattice origin o) at every grid node (i hx, j hy, k hz) into V[nz][ny][nx] (FP64).
// The lattice position of a node separates over the axes: interp_axes_kernel
// tabulates, per axis, the two bracketing lattice indices (wrapped) and the fraction.
struct AxisPos {
    int i0, i1;
    double f;
};

struct InterpArgs {
    double h[3], L[3], o[3];
    int n[3], c[3];
};

__global__ void interp_axes_kernel(InterpArgs A, AxisPos *__restrict__ tab)
{
    const int total = A.n[0] + A.n[1] + A.n[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const int a = t < A.n[0] ? 0 : t < A.n[0] + A.n[1] ? 1 : 2;
        const int i = t - (a == 0 ? 0 : a == 1 ? A.n[0] : A.n[0] + A.n[1]);
        const int n = A.c[a];
        const double u = (i * A.h[a] - A.o[a]) / A.L[a] * n;
        const double fl = floor(u);
        long long k = static_cast<long long>(fl) % n;
        if (k < 0) k += n;
        AxisPos p;
        p.f = u - fl;
        p.i0 = static_cast<int>(k);
        p.i1 = p.i0 + 1 == n ? 0 : p.i0 + 1;
        tab[t] = p;
    }
}

__global__ void interp_kernel(int nx, int ny, int nz, const double *__restrict__ Vc, int cnx,
                              int cny, const AxisPos *__restrict__ tab, double *__restrict__ V)
{
    for_each_node(nx, ny, nz, [&](int x, int y, int z, long long t) {
        const AxisPos px = tab[x], py = tab[nx + y], pz = tab[nx + ny + z];
        auto at = [&](int k, int j, int i) {
            return Vc[(static_cast<long long>(k) * cny + j) * cnx + i];
        };
        const double fx = px.f, fy = py.f, fz = pz.f;
        const double c00 = at(pz.i0, py.i0, px.i0) * (1 - fx) + at(pz.i0, py.i0, px.i1) * fx;
        const double c01 = at(pz.i0, py.i1, px.i0) * (1 - fx) + at(pz.i0, py.i1, px.i1) * fx;
        const double c10 = at(pz.i1, py.i0, px.i0) * (1 - fx) + at(pz.i1, py.i0, px.i1) * fx;
        const double c11 = at(pz.i1, py.i1, px.i0) * (1 - fx) + at(pz.i1, py.i1, px.i1) * fx;
        const double c0 = c00 * (1 - fy) + c01 * fy;
        const double c1 = c10 * (1 - fy) + c11 * fy;
        V[t] = c0 * (1 - fz) + c1 * fz;
    });
}

size_t interp_scratch_bytes(const MemberDev &m)
{
    return (static_cast<size_t>(m.nx) + m.ny + m.nz) * sizeof(AxisPos);
}

cudaError_t launch_interp(const MemberDev &m, double hx, double hy, double hz, const double *Vc,
                          int cnx, int cny, int cnz, const double L[3], const double o[3],
                          void *scratch, double *V, cudaStream_t s)
{
    InterpArgs A;
    const double h[3] = {hx, hy, hz};
    const int n[3] = {m.nx, m.ny, m.nz}, c[3] = {cnx, cny, cnz};
    for (int a = 0; a < 3; ++a) {
        A.h[a] = h[a];
        A.L[a] = L[a];
        A.o[a] = o[a];
        A.n[a] = n[a];
        A.c[a] = c[a];
    }
    AxisPos *tab = static_cast<AxisPos *>(scratch);
    const int total = m.nx + m.ny + m.nz;
    interp_axes_kernel<<<(total + kThreads - 1) / kThreads, kThreads, 0, s>>>(A, tab);
    const NodeLaunch Ln = node_launch(m);
    interp_kernel<<<Ln.grid, Ln.threads, 0, s>>>(m.nx, m.ny, m.nz, Vc, cnx, cny, tab, V);
    return cudaGetLastError();
}

void observables_shape(const MemberDev &m, int precision, int *nparts_out, int *zch_out)
{
    const int vec = precision == 0 ? 2 : 4;          // one 16-byte vector per field and plane
    const bool vector = m.nx % vec == 0;
    const long long groups = static_cast<long long>(vector ? m.nx / vec : m.nx) * m.ny;
    // z planes per work item: kObsZ on large grids; fewer (down to kObsZmin) where
    // that would leave less than about one item per thread of kObsParts blocks, since
    // a thread marches its planes one after the other (a 96 x 96 x 192 member: 16).
    // Each item also reads the planes on either side of its chunk, so shorter chunks
    // read more: 16 planes read 18.
    const long long want = (static_cast<long long>(kObsParts) * kObsThreads + groups - 1) / groups;
    const int zch = static_cast<int>(
        std::min<long long>(kObsZ, std::max<long long>(kObsZmin, (m.nz + want - 1) / want)));
    const long long nitems = groups * ((m.nz + zch - 1) / zch);
    *zch_out = zch;
    *nparts_out = static_cast<int>(
        std::max<long long>(1, std::min<long long>((nitems + kObsThreads - 1) / kObsThreads, kObsParts)));
}

cudaError_t launch_observables_batch(const MemberDev *members, const ObsSlice *slices, int nmembers,
                                     int total_blocks, int precision, int buf, double *partials,
                                     double *records, long long rec_stride, int *status, long long step,
                                     cudaStream_t s)
{
    // every member's nx is a multiple of 4, so the vector form applies to all
    if (precision == 0)
        observables_batch_kernel<double, 2><<<total_blocks, kObsThreads, 0, s>>>(members, slices, nmembers,
                                                                                 buf, partials);
    else
        observables_batch_kernel<float, 4><<<total_blocks, kObsThreads, 0, s>>>(members, slices, nmembers,
                                                                                buf, partials);
    observables_batch_finalize_kernel<<<nmembers, kThreads, 0, s>>>(members, slices, partials, records,
                                                                    rec_stride, status, step);
    return cudaGetLastError();
}

cudaError_t launch_observables(const MemberDev &m, int precision, int buf, double *partials,
                               double *record, int *status, double q_ref, long long step,
                               cudaStream_t s)
{
    const int vec = precision == 0 ? 2 : 4;
    const bool vector = m.nx % vec == 0;
    int nparts = 0, zch = 0;
    observables_shape(m, precision, &nparts, &zch);
    auto run = [&](auto kernel_full, auto kernel_short) {
        if (zch == kObsZ) kernel_full<<<nparts, kObsThreads, 0, s>>>(m, buf, partials, zch);
        else kernel_short<<<nparts, kObsThreads, 0, s>>>(m, buf, partials, zch);
    };
    if (precision == 0) {
        if (vector) run(observables_kernel<double, 2, kObsZ>, observables_kernel<double, 2, 0>);
        else run(observables_kernel<double, 1, kObsZ>, observables_kernel<double, 1, 0>);
    } else {
        if (vector) run(observables_kernel<float, 4, kObsZ>, observables_kernel<float, 4, 0>);
        else run(observables_kernel<float, 1, kObsZ>, observables_kernel<float, 1, 0>);
    }
    observables_finalize_kernel<<<1, kThreads, 0, s>>>(m, partials, nparts, record, status, q_ref,
                                                       step);
    return cudaGetLastError();
}

}  // namespace tdse
