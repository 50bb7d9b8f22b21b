// Device helpers shared by the fused-step kernels: mbarrier and TMA wrappers,
// vector shared/global access, correctly rounded and paired FP32 arithmetic,
// the compile-time kernel shape and the per-item scalars.
#pragma once

#include <atomic>
#include <cstdint>

#include "tdse_internal.cuh"

namespace tdse {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s: drain of loads in flight

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

__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Non-blocking test of the phase.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait: false if the phase did not complete within limit_ns.  A limit of
// 0 tests the phase once without waiting, so that a wait for a load still in
// flight expires (the host's way of exercising the expiry path with valid loads).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs)
{
    if (limit_ns == 0) return mbar_test_wait(bar, parity);
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as another warp has raised *abort_flag:
// 1 the phase completed, 0 the limit expired, -1 abandoned (flag raised).  A limit
// of 0 tests the phase once, as in mbar_wait_bounded.
__device__ __forceinline__ int mbar_wait_or_abort(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns,
                                                  const volatile int *abort_flag)
{
    if (limit_ns == 0) return mbar_test_wait(bar, parity) ? 1 : 0;
    if (mbar_try_wait(bar, parity)) return 1;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return -1;
        if (global_ns() - t0 > limit_ns) return 0;
    }
    return 1;
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

// Global store of one vector with the streaming hint (st.global.cs: evicted first),
// for output planes that this launch never reads back.
template <typename Real>
__device__ __forceinline__ void st_vec_stream(Real *p, const Real (&v)[VecOf<Real>::N]);
template <>
__device__ __forceinline__ void st_vec_stream<float>(float *p, const float (&v)[4])
{
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
}
template <>
__device__ __forceinline__ void st_vec_stream<double>(double *p, const double (&v)[2])
{
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
}

// Rounded product that the compiler may not fuse into a following add: the
// absorbing factor must round identically whether its product is stored
// (one step per launch) or consumed in registers (several steps per launch).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// Paired FP32 arithmetic (one instruction for two lanes, each lane rounded to
// nearest exactly as the scalar operation).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Compile-time shape of one fused-step kernel.
//   H     half-step stages per launch (2T)
//   TPX   threads across a region row (VEC cells each)
//   ROWS  region rows; each thread owns RPT consecutive rows
//   PF    planes loaded ahead of use
//   DSTASH  d is copied out of shared memory as each plane lands (tensor-memory
//           kernel), so its ring only covers the planes in flight
//   OWNRINGS  the kernel lays out its own rings (and checks their size itself); SMEM
//           below is then only the layout of the other kernels
template <typename Real_, int H_, int TPX_, int ROWS_, int RPT_, bool KAHAN_, int PF_, int MINB_ = 1,
          bool DSTASH_ = false, bool OWNRINGS_ = false>
struct Cfg {
    typedef Real_ Real;
    static constexpr int H = H_, TPX = TPX_, ROWS = ROWS_, RPT = RPT_, PF = PF_;
    static constexpr int MINB = MINB_;                  // CTAs resident per SM
    static constexpr bool KAHAN = KAHAN_;
    static constexpr int VEC = VecOf<Real>::N;
    static constexpr int W = VEC * TPX;                 // region width (elements)
    static constexpr int AX = 16 / static_cast<int>(sizeof(Real));
    static constexpr int HX = (H + AX - 1) / AX * AX;   // x halo, TMA-aligned
    static constexpr int TX = W - 2 * HX;
    static constexpr int TY = ROWS - 2 * H;
    static constexpr int NT = TPX * ROWS / RPT;
    static constexpr bool ROW_IN_WARP = 32 % TPX == 0;  // every region row sits inside one warp
    static constexpr int RW = ROW_IN_WARP ? 32 / TPX * RPT : 0;   // rows per warp
    static constexpr int PLANE = W * ROWS;
    static constexpr int PLANE_BYTES = PLANE * static_cast<int>(sizeof(Real));
    static constexpr int NFC = KAHAN ? 2 : 1;           // a field (and its compensation) per slot
    static constexpr int NR = PF + 3;                   // R ring: read up to two planes back
    static constexpr int NI = PF + 2;                   // I ring: read one plane back
    static constexpr bool DSTASH = DSTASH_;
    static constexpr int ND = DSTASH ? PF + 1 : PF + H + 1;   // d is read H planes back
    static constexpr int NB = PF + 1;
    static constexpr int NSB = 2 * (H - 1);             // stage planes, double-buffered
    static constexpr int NPLANES = (NR + NI) * NFC + ND + NSB;
    static constexpr size_t SMEM = static_cast<size_t>(NPLANES) * PLANE_BYTES + 8 * NB + 128;
    static constexpr uint32_t TX_BYTES = PLANE_BYTES * (2 * NFC + 1);
    static_assert(TPX <= 32 && NT % 32 == 0, "whole warps");
    static_assert(ROWS % RPT == 0, "rows per thread must divide the region");
    static_assert(TX > 0 && TY > 0, "halo larger than region");
    static_assert(W <= 256 && ROWS <= 256, "TMA box dimension limit");
    static_assert(H % 2 == 0, "whole time steps only");
    static_assert(OWNRINGS_ || SMEM <= 232448, "more than 227 KB of shared memory per CTA");
    static_assert(OWNRINGS_ || MINB * (SMEM + 1024) <= 233472, "CTAs per SM exceed the shared memory");
};

// One row of an FP32 stage update in paired instructions: the increment
// delta = A f = cx (f[x-1] + f[x+1]) + cy (f[y-1] + f[y+1]) + cz (f[z-1] + f[z+1]) + d f
// at the row's VEC cells, then out = acc + delta (odd stage, Eq. 9) or
// out = acc - delta (even stage, Eq. 8).  With KAHAN the accumulation carries the
// compensation term: odd: y = delta - c, t = acc + y, c' = (t - acc) - y;
// even (increment -delta): with y' = delta + c = -y exactly, t = acc - y',
// c' = (t - acc) + y'.  Only the x-neighbour sum, whose operands are shifted by
// one lane, is scalar.  xl / xr are the row's outer x neighbours, ylo / yhi the
// rows below / above.
template <bool KAHAN, int VEC>
__device__ __forceinline__ void update_row_f32(bool odd, const float (&c)[VEC], float xl, float xr,
                                               const float (&ylo)[VEC], const float (&yhi)[VEC],
                                               const float (&zm)[VEC], const float (&zp)[VEC],
                                               const float (&dd)[VEC], const float (&acc)[VEC],
                                               const float (&cacc)[VEC], float2 cx2, float2 cy2,
                                               float2 cz2, float (&out)[VEC], float (&cout)[VEC])
{
    auto pr = [](const float *a, int i) { return make_float2(a[i], a[i + 1]); };
#pragma unroll
    for (int v = 0; v < VEC; v += 2) {
        const float2 sx = make_float2((v == 0 ? xl : c[v - 1]) + c[v + 1],
                                      c[v] + (v + 2 == VEC ? xr : c[v + 2]));
        const float2 sy = add2(pr(ylo, v), pr(yhi, v));
        const float2 sz = add2(pr(zm, v), pr(zp, v));
        float2 delta = mul2(pr(dd, v), pr(c, v));
        delta = fma2(cz2, sz, delta);
        delta = fma2(cy2, sy, delta);
        delta = fma2(cx2, sx, delta);
        const float2 a = pr(acc, v);
        float2 o;
        if constexpr (KAHAN) {
            const float2 ca = pr(cacc, v);
            float2 co;
            if (odd) {
                const float2 y = sub2(delta, ca);
                o = add2(a, y);
                co = sub2(sub2(o, a), y);
            } else {
                const float2 y = add2(delta, ca);
                o = sub2(a, y);
                co = add2(sub2(o, a), y);
            }
            cout[v] = co.x;
            cout[v + 1] = co.y;
        } else {
            o = odd ? add2(a, delta) : sub2(a, delta);
        }
        out[v] = o.x;
        out[v + 1] = o.y;
    }
}

// Per-item scalars staged in shared memory by thread 0.
struct ItemScalars {
    void *outR, *outI, *outCR, *outCI, *mask;
    double *flux, *jlast;
    long long plane, pitch;
    double cx, cy, cz, cj, dt;
    int m, tile_x, tile_y, kz0, kz1, nx, ny, nz, G;
    int per_x, per_y, per_z, det_k, mask_lo, mask_hi;
};

// Thread 0 of a fused-step CTA: take the next work item (member, xy tile, z-chunk)
// from the counter into *item and, if there is one, stage the member's scalars in
// shared memory (loop invariants then never come back from global memory).
__device__ __forceinline__ void fetch_item(const MemberDev *__restrict__ members,
                                           const WorkDev *__restrict__ work, int *counter,
                                           int in_buf, int *item, ItemScalars &S)
{
    const int it_ = atomicAdd(counter, 1);
    *item = it_;
    if (it_ >= work->total) return;
    int mm = 0;
    while (it_ >= work->item_begin[mm + 1]) ++mm;
    const MemberDev &Mm = members[mm];
    const int local = it_ - work->item_begin[mm];
    const int ntx = work->tiles_x[mm], nty = work->tiles_y[mm];
    S.m = mm;
    S.tile_x = local % ntx;
    S.tile_y = (local / ntx) % nty;
    S.kz0 = (local / (ntx * nty)) * work->chunk[mm];
    S.kz1 = min(S.kz0 + work->chunk[mm], Mm.nz);
    S.nx = Mm.nx; S.ny = Mm.ny; S.nz = Mm.nz; S.G = Mm.G;
    S.per_x = Mm.per_x; S.per_y = Mm.per_y; S.per_z = Mm.per_z;
    S.det_k = Mm.det_k; S.mask_lo = Mm.mask_lo; S.mask_hi = Mm.mask_hi;
    S.pitch = Mm.pitch; S.plane = Mm.plane;
    S.cx = Mm.cx; S.cy = Mm.cy; S.cz = Mm.cz; S.cj = Mm.cj; S.dt = Mm.dt;
    S.mask = Mm.mask; S.flux = Mm.flux; S.jlast = Mm.jlast;
    S.outR = Mm.R[1 - in_buf]; S.outI = Mm.I[1 - in_buf];
    S.outCR = Mm.cR[1 - in_buf]; S.outCI = Mm.cI[1 - in_buf];
}

// One output row of the last stage at offset o of the padded arrays: R, I (and the
// compensation terms), plus the ghost copies of periodic axes when the row touches
// a seam (both sides when an axis is shorter than twice the ghost width).  The
// stores are marked evict-first: this launch never reads its output planes, and in
// L2 they would displace input planes whose halos neighbouring tiles still read.
template <typename Real, bool KAHAN, int VEC>
__device__ __forceinline__ void store_output_row(const ItemScalars &S, Real *outR, Real *outI,
                                                 Real *outCR, Real *outCI, long long o,
                                                 long long pitch, bool seam, int xs, int y,
                                                 const Real (&r)[VEC], const Real (&i)[VEC],
                                                 const Real (&cr)[VEC], const Real (&ci)[VEC])
{
    auto st_out = [](Real *p, const Real (&v)[VEC]) { st_vec_stream<Real>(p, v); };
    st_out(outR + o, r);
    st_out(outI + o, i);
    if constexpr (KAHAN) {
        st_out(outCR + o, cr);
        st_out(outCI + o, ci);
    }
    if (!seam) return;
    const int G = S.G, nx = S.nx, ny = S.ny;
    int dxs[3] = {0, 0, 0}, dys[3] = {0, 0, 0};
    int ndx = 1, ndy = 1;
    if (S.per_x) {
        if (xs < G) dxs[ndx++] = nx;
        if (xs >= nx - G) dxs[ndx++] = -nx;
    }
    if (S.per_y) {
        if (y < G) dys[ndy++] = ny;
        if (y >= ny - G) dys[ndy++] = -ny;
    }
    for (int a = 0; a < ndy; ++a)
        for (int b = 0; b < ndx; ++b) {
            if (a == 0 && b == 0) continue;
            const long long og = o + dys[a] * pitch + dxs[b];
            st_out(outR + og, r);
            st_out(outI + og, i);
            if constexpr (KAHAN) {
                st_out(outCR + og, cr);
                st_out(outCI + og, ci);
            }
        }
}

}  // namespace

// Dynamic shared memory above 48 KB must be allowed per kernel, and the setting
// belongs to the device that is current when it is made: set it once on each
// device (a process may drive several GPUs, one context on each).
template <class K>
cudaError_t allow_dynamic_smem(K *kernel, size_t bytes, std::atomic<uint64_t> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? (uint64_t{1} << dev) : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

}  // namespace tdse
