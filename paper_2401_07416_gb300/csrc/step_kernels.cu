// Fused leapfrog step for the 3-D TDSE (arXiv 2401.07416, Sec. 2.1, Eqs. 8-9).
//
// One CTA owns an xy tile of TX x TY output columns and a z-chunk [kz0, kz1) of
// output planes, and marches along z.  It runs the 2T half-steps of T fused time
// steps as a pipeline of stages s = 1..2T: odd stages apply Eq. 9
// (I += A R), even stages Eq. 8 (R -= A I) followed by the absorbing factor.
// Stage s works on plane p - s while plane p is being loaded, so every stage
// reads its z-neighbours from a three-plane register window of the previous
// stage's output (old = q-1, center = q, new = q+1) and its x/y-neighbours from
// the previous stage's center plane in shared memory (y) or by warp shuffles (x).
//
// Input planes of R, I, d (and the Kahan compensation terms) arrive by TMA
// (cp.async.bulk.tensor.3d) into shared-memory rings PF planes ahead of use,
// completed on mbarriers.  Each stage's output is valid on a region that
// shrinks by one cell per stage, so a tile loads a halo of 2T cells in y and
// 2T rounded up to 16 bytes in x.  The ghost zones of periodic axes make every
// tile load a single box.  Outputs go to the other ping-pong buffer with
// coalesced vector stores (plus the ghost copies of periodic axes).
//
// HBM traffic per fused launch: R, I, d read once and R, I written once per
// node (FP32: 20 bytes, FP64: 40 bytes; Kahan adds 16 bytes), i.e. 20/T bytes
// per node-update in FP32.
#include <cstdio>

#include "tdse_internal.cuh"

namespace tdse {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per barrier wait

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: false if the phase did not complete within kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y,
                                            int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <typename Real>
struct VecOf;
template <>
struct VecOf<float> {
    typedef float4 type;
    static constexpr int N = 4;
};
template <>
struct VecOf<double> {
    typedef double2 type;
    static constexpr int N = 2;
};

template <typename Real>
__device__ __forceinline__ void ld_vec(const Real *p, Real (&v)[VecOf<Real>::N]);
template <>
__device__ __forceinline__ void ld_vec<float>(const float *p, float (&v)[4])
{
    float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld_vec<double>(const double *p, double (&v)[2])
{
    double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x; v[1] = t.y;
}
template <typename Real>
__device__ __forceinline__ void st_vec(Real *p, const Real (&v)[VecOf<Real>::N]);
template <>
__device__ __forceinline__ void st_vec<float>(float *p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_vec<double>(double *p, const double (&v)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

// Rounded product that the compiler may not fuse into a following add: the
// absorbing factor must round identically whether its product is stored
// (one step per launch) or consumed in registers (several steps per launch).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Compile-time shape of one fused-step kernel.
template <typename Real_, int H_, int TPX_, int ROWS_, bool KAHAN_, int PF_>
struct Cfg {
    typedef Real_ Real;
    static constexpr int H = H_;          // half-step stages per launch (2T)
    static constexpr int TPX = TPX_;      // threads per region row
    static constexpr int ROWS = ROWS_;    // region rows (one per thread row)
    static constexpr bool KAHAN = KAHAN_;
    static constexpr int PF = PF_;        // planes loaded ahead
    static constexpr int VEC = VecOf<Real>::N;
    static constexpr int W = VEC * TPX;   // region width (elements)
    static constexpr int AX = 16 / static_cast<int>(sizeof(Real));
    static constexpr int HX = (H + AX - 1) / AX * AX;   // x halo, TMA-aligned
    static constexpr int TX = W - 2 * HX;
    static constexpr int TY = ROWS - 2 * H;
    static constexpr int NT = TPX * ROWS;
    static constexpr int RW = 32 / TPX;   // rows per warp
    static constexpr int NR = PF + 2, NI = PF + 2, ND = PF + H + 1;
    static constexpr int NCR = KAHAN ? PF + 3 : 0, NCI = KAHAN ? PF + 2 : 0;
    static constexpr int NCRm = KAHAN ? NCR : 1, NCIm = KAHAN ? NCI : 1;   // modulus-safe
    static constexpr int NB = PF + 1;
    static constexpr int PLANE = W * ROWS;
    static constexpr int PLANE_BYTES = PLANE * static_cast<int>(sizeof(Real));
    static constexpr int NSB = 2 * (H - 1);
    static constexpr int NPLANES = NR + NI + ND + NCR + NCI + NSB;
    static constexpr size_t SMEM = static_cast<size_t>(NPLANES) * PLANE_BYTES + 8 * NB + 128;
    static constexpr uint32_t TX_BYTES = PLANE_BYTES * (KAHAN ? 5 : 3);
    static_assert(TPX <= 32 && 32 % TPX == 0, "a region row must sit inside one warp");
    static_assert(TX > 0 && TY > 0, "halo larger than region");
    static_assert(W <= 256 && ROWS <= 256, "TMA box dimension limit");
    static_assert(H % 2 == 0, "whole time steps only");
};

template <class C>
__global__ void __launch_bounds__(C::NT, 1)
    fused_step_kernel(const MemberDev *__restrict__ members, const WorkDev *__restrict__ work,
                      int *counter, int *status, int in_buf)
{
    typedef typename C::Real Real;
    constexpr int H = C::H, VEC = C::VEC, W = C::W, ROWS = C::ROWS, PLANE = C::PLANE;
    constexpr int NB = C::NB, PF = C::PF;

    extern __shared__ unsigned char smem_raw[];
    Real *base = reinterpret_cast<Real *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                          ~static_cast<uintptr_t>(127));
    Real *ringR = base;
    Real *ringI = ringR + C::NR * PLANE;
    Real *ringD = ringI + C::NI * PLANE;
    Real *ringCR = ringD + C::ND * PLANE;
    Real *ringCI = ringCR + C::NCR * PLANE;
    Real *sbuf = ringCI + C::NCI * PLANE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbuf + C::NSB * PLANE);
    __shared__ int s_item;

    const int tid = threadIdx.x;
    const int row = tid / C::TPX;
    const int qx = tid % C::TPX;
    const int warp_row0 = (tid & ~31) / C::TPX;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    long long gbase = 0;   // loads issued by this CTA before the current item
    bool aborted = false;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= work->total) break;
        int m = 0;
        while (item >= work->item_begin[m + 1]) ++m;
        const MemberDev &M = members[m];
        const int local = item - work->item_begin[m];
        const int ntx = work->tiles_x[m], nty = work->tiles_y[m];
        const int tile_x = local % ntx;
        const int tile_y = (local / ntx) % nty;
        const int kz0 = (local / (ntx * nty)) * work->chunk[m];
        const int kz1 = min(kz0 + work->chunk[m], M.nz);
        const int L0 = kz0 - H;                 // first plane loaded
        const int nit = (kz1 - kz0) + 2 * H;    // iterations (planes loaded)
        const int G = M.G, nx = M.nx, ny = M.ny, nz = M.nz;
        const int bx = G + tile_x * C::TX - C::HX;   // padded coordinates of the box
        const int by = G + tile_y * C::TY - H;
        const int xs = tile_x * C::TX - C::HX + qx * VEC;  // unpadded x of this thread's first cell
        const int ys = tile_y * C::TY - H + row;
        const bool zper = M.per_z != 0;
        const Real cx = static_cast<Real>(M.cx), cy = static_cast<Real>(M.cy),
                   cz = static_cast<Real>(M.cz);
        const Real *maskz = reinterpret_cast<const Real *>(M.mask);
        Real *outR = reinterpret_cast<Real *>(M.R[1 - in_buf]);
        Real *outI = reinterpret_cast<Real *>(M.I[1 - in_buf]);
        Real *outCR = reinterpret_cast<Real *>(M.cR[1 - in_buf]);
        Real *outCI = reinterpret_cast<Real *>(M.cI[1 - in_buf]);

        // Cells outside the domain on a walled axis are kept at zero after every stage.
        const bool walls = (!M.per_x && (xs < 0 || xs + VEC > nx)) || (!M.per_y && (ys < 0 || ys >= ny));
        Real keep[VEC];
#pragma unroll
        for (int v = 0; v < VEC; ++v) {
            const bool in_x = M.per_x || (xs + v >= 0 && xs + v < nx);
            const bool in_y = M.per_y || (ys >= 0 && ys < ny);
            keep[v] = (in_x && in_y) ? Real(1) : Real(0);
        }
        const bool store_cell = row >= H && row < H + C::TY && qx * VEC >= C::HX &&
                                qx * VEC < C::HX + C::TX && ys < ny && xs < nx;
        const int kd = M.det_k;
        const bool flux_owner = kd >= kz0 && kd < kz1;

        // Register windows of the stage outputs F_0 .. F_{H-1}: [0] old (q-1),
        // [1] center (q), [2] new (q+1); Kahan compensation windows alongside.
        Real w[H][3][VEC];
        Real cw[H][3][VEC];
#pragma unroll
        for (int f = 0; f < H; ++f)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    w[f][k][v] = Real(0);
                    cw[f][k][v] = Real(0);
                }

        auto issue = [&](int l) {
            const int L = L0 + l;
            const int zc = zper ? ((L % nz) + nz) % nz : L;
            uint64_t *bar = &bars[(gbase + l) % NB];
            mbar_arrive_expect_tx(bar, C::TX_BYTES);
            tma_load_3d(ringR + (l % C::NR) * PLANE, &M.tm_R[in_buf], bx, by, zc, bar);
            tma_load_3d(ringI + (l % C::NI) * PLANE, &M.tm_I[in_buf], bx, by, zc, bar);
            tma_load_3d(ringD + (l % C::ND) * PLANE, &M.tm_d, bx, by, zc, bar);
            if (C::KAHAN) {
                tma_load_3d(ringCR + (l % C::NCRm) * PLANE, &M.tm_cR[in_buf], bx, by, zc, bar);
                tma_load_3d(ringCI + (l % C::NCIm) * PLANE, &M.tm_cI[in_buf], bx, by, zc, bar);
            }
        };

        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int l = 0; l < PF && l < nit; ++l) issue(l);
        }

        int issued = min(PF, nit);
        int waited = 0;   // loads consumed by this thread
        for (int it = 0; it < nit; ++it) {
            const int p = L0 + it;
            if (__syncthreads_or(aborted ? 1 : 0)) {
                aborted = true;
                break;
            }
            if (tid == 0 && it + PF < nit) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                issue(it + PF);
            }
            if (it + PF < nit) issued = it + PF + 1;
            if (!mbar_wait_bounded(&bars[(gbase + it) % NB],
                                   static_cast<uint32_t>(((gbase + it) / NB) & 1))) {
                atomicOr(status, 1);
                aborted = true;
                continue;
            }
            waited = it + 1;

            // stage 0: R of plane p enters the window of F_0
            {
                Real nr[VEC];
                ld_vec<Real>(ringR + (it % C::NR) * PLANE + row * W + qx * VEC, nr);
                const bool oob = !zper && (p < 0 || p >= nz);
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    w[0][0][v] = w[0][1][v];
                    w[0][1][v] = w[0][2][v];
                    w[0][2][v] = oob ? Real(0) : nr[v];
                }
            }

#pragma unroll
            for (int s = 1; s <= H; ++s) {
                const int q = p - s;
                if (it < 2 * s) continue;                                     // pipeline filling
                if (warp_row0 + C::RW <= s || warp_row0 >= ROWS - s) continue;  // rows outside the cone
                const bool odd = (s & 1) != 0;
                const bool q_out = !zper && (q < 0 || q >= nz);
                const int qm = zper ? ((q % nz) + nz) % nz : q;
                const Real mq = q_out ? Real(0) : maskz[qm];

                // stencil input F_{s-1}: center plane in shared memory for the y-neighbours
                const Real *S = (s == 1) ? ringR + ((it - 1) % C::NR) * PLANE
                                         : sbuf + ((s - 2) * 2 + ((it - 1) & 1)) * PLANE;
                const int rm = row > 0 ? row - 1 : row;
                const int rp = row < ROWS - 1 ? row + 1 : row;
                Real ym[VEC], yp[VEC], dd[VEC];
                ld_vec<Real>(S + rm * W + qx * VEC, ym);
                ld_vec<Real>(S + rp * W + qx * VEC, yp);
                ld_vec<Real>(ringD + ((it - s) % C::ND) * PLANE + row * W + qx * VEC, dd);
                const Real xl = __shfl_up_sync(kFull, w[s - 1][1][VEC - 1], 1);
                const Real xr = __shfl_down_sync(kFull, w[s - 1][1][0], 1);

                // accumulator: the field of stage s-2 at plane q
                Real acc[VEC], cacc[VEC];
                if (s == 1) {
                    ld_vec<Real>(ringI + ((it - 1) % C::NI) * PLANE + row * W + qx * VEC, acc);
                    if (C::KAHAN)
                        ld_vec<Real>(ringCI + ((it - 1) % C::NCIm) * PLANE + row * W + qx * VEC, cacc);
                } else {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        acc[v] = w[s - 2][0][v];
                        cacc[v] = cw[s - 2][0][v];
                    }
                    if (s == 2 && C::KAHAN)
                        ld_vec<Real>(ringCR + ((it - 2) % C::NCRm) * PLANE + row * W + qx * VEC, cacc);
                    if (odd) {   // I of the previous step still carries its absorbing factor
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            acc[v] = mul_rn(acc[v], mq);
                            cacc[v] = mul_rn(cacc[v], mq);
                        }
                    }
                }

                Real out[VEC], cout[VEC];
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const Real c0 = w[s - 1][1][v];
                    const Real sx = (v == 0 ? xl : w[s - 1][1][v - 1]) +
                                    (v == VEC - 1 ? xr : w[s - 1][1][v + 1]);
                    const Real sy = ym[v] + yp[v];
                    const Real sz = w[s - 1][0][v] + w[s - 1][2][v];
                    const Real delta = fma(cx, sx, fma(cy, sy, fma(cz, sz, dd[v] * c0)));
                    const Real inc = odd ? delta : -delta;
                    if (C::KAHAN) {
                        const Real y = inc - cacc[v];
                        const Real t = acc[v] + y;
                        cout[v] = (t - acc[v]) - y;
                        out[v] = t;
                    } else {
                        out[v] = acc[v] + inc;
                        cout[v] = Real(0);
                    }
                    if (!odd) {          // Eq. 8 step complete: absorbing factor on R
                        out[v] = mul_rn(out[v], mq);
                        cout[v] = mul_rn(cout[v], mq);
                    }
                    if (walls) {
                        out[v] *= keep[v];
                        cout[v] *= keep[v];
                    }
                    if (q_out) {
                        out[v] = Real(0);
                        cout[v] = Real(0);
                    }
                }

                // detector flux of step (s+1)/2: R at planes kd, kd+1 and the new I
                if (odd && flux_owner && q == kd + 1 && store_cell) {
                    const int pix = ys * nx + xs;
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        const double j = M.cj * (static_cast<double>(w[s - 1][0][v]) * out[v] -
                                                 static_cast<double>(w[s - 1][1][v]) * w[s][2][v]);
                        M.flux[pix + v] += j * M.dt;
                        if (s == H - 1) M.jlast[pix + v] = j;
                    }
                }

                if (s < H) {
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        w[s][0][v] = w[s][1][v];
                        w[s][1][v] = w[s][2][v];
                        w[s][2][v] = out[v];
                        cw[s][0][v] = cw[s][1][v];
                        cw[s][1][v] = cw[s][2][v];
                        cw[s][2][v] = cout[v];
                    }
                    st_vec<Real>(sbuf + ((s - 1) * 2 + (it & 1)) * PLANE + row * W + qx * VEC, out);
                } else if (store_cell && q >= kz0 && q < kz1) {
                    Real vi[VEC], vci[VEC];
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        vi[v] = mul_rn(w[H - 1][1][v], mq);
                        vci[v] = mul_rn(cw[H - 1][1][v], mq);
                    }
                    // primary location plus the ghost copies of periodic axes
                    int xo[2] = {xs, xs};
                    int yo[2] = {ys, ys};
                    int nxo = 1, nyo = 1;
                    if (M.per_x) {
                        if (xs < G) xo[nxo++] = xs + nx;
                        else if (xs >= nx - G) xo[nxo++] = xs - nx;
                    }
                    if (M.per_y) {
                        if (ys < G) yo[nyo++] = ys + ny;
                        else if (ys >= ny - G) yo[nyo++] = ys - ny;
                    }
                    const long long zoff = static_cast<long long>(q) * M.plane;
                    for (int a = 0; a < nyo; ++a)
                        for (int b = 0; b < nxo; ++b) {
                            const long long o = zoff + static_cast<long long>(yo[a] + G) * M.pitch + (xo[b] + G);
                            st_vec<Real>(outR + o, out);
                            st_vec<Real>(outI + o, vi);
                            if (C::KAHAN) {
                                st_vec<Real>(outCR + o, cout);
                                st_vec<Real>(outCI + o, vci);
                            }
                        }
                }
            }
        }

        if (__syncthreads_or(aborted ? 1 : 0)) {
            // wait (bounded) for the loads still in flight, then leave
            if (tid == 0) {
                for (int l = waited; l < issued; ++l)
                    mbar_wait_bounded(&bars[(gbase + l) % NB],
                                      static_cast<uint32_t>(((gbase + l) / NB) & 1));
            }
            __syncthreads();
            return;
        }
        gbase += nit;
        __syncthreads();
    }
}

template <class C>
cudaError_t launch_cfg(const StepLaunch &L)
{
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(fused_step_kernel<C>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(C::SMEM));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    fused_step_kernel<C><<<L.grid, C::NT, C::SMEM, L.stream>>>(L.members, L.work, L.counter,
                                                               L.status, L.in_buf);
    return cudaGetLastError();
}

template <class C>
void fill_config(StepConfig *cfg)
{
    cfg->tile_x = C::TX;
    cfg->tile_y = C::TY;
    cfg->box_x = C::W;
    cfg->box_y = C::ROWS;
    cfg->threads = C::NT;
    cfg->smem = C::SMEM;
    cfg->ctas_per_sm = 1;
}

// The kernel configurations of the library.
typedef Cfg<float, 2, 16, 32, false, 2> F32T1;
typedef Cfg<float, 2, 16, 32, true, 2> K32T1;
typedef Cfg<float, 4, 16, 32, false, 2> F32T2;
typedef Cfg<float, 4, 16, 28, true, 2> K32T2;
typedef Cfg<double, 2, 32, 24, false, 1> F64T1;

}  // namespace

bool step_config(int precision, int tsteps, StepConfig *cfg)
{
    if (precision == 0 && tsteps == 1) { fill_config<F64T1>(cfg); return true; }
    if (precision == 1 && tsteps == 1) { fill_config<F32T1>(cfg); return true; }
    if (precision == 1 && tsteps == 2) { fill_config<F32T2>(cfg); return true; }
    if (precision == 2 && tsteps == 1) { fill_config<K32T1>(cfg); return true; }
    if (precision == 2 && tsteps == 2) { fill_config<K32T2>(cfg); return true; }
    return false;
}

cudaError_t launch_step(int precision, int tsteps, const StepLaunch &L)
{
    if (precision == 0 && tsteps == 1) return launch_cfg<F64T1>(L);
    if (precision == 1 && tsteps == 1) return launch_cfg<F32T1>(L);
    if (precision == 1 && tsteps == 2) return launch_cfg<F32T2>(L);
    if (precision == 2 && tsteps == 1) return launch_cfg<K32T1>(L);
    if (precision == 2 && tsteps == 2) return launch_cfg<K32T2>(L);
    return cudaErrorInvalidValue;
}

}  // namespace tdse
