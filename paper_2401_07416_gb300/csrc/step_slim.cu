// Fused leapfrog step, tensor-memory windows, with every ring slot a compile-time
// offset (arXiv 2401.07416, Sec. 2.1, Eqs. 8-9), FP32 and FP32 + Kahan, two time
// steps per launch.
//
// Same schedule, windows and arithmetic as fused_step_tmem_kernel (step_tmem.cu):
// a CTA marches an xy tile along z, stage s of the 2T half-step stages works on
// plane p - s while plane p arrives by TMA, the stage windows and d live in tensor
// memory.  What differs is the bookkeeping, which dominated the instruction count
// there (ring heads, window phases, d slots and their addresses were computed at
// run time, about a third of all instructions):
//   - Fields read only by the thread that owns a cell are loaded late: the loads
//     that complete on the barrier of plane p bring R and d at p, I and cI at p-1
//     and cR at p-2, so their rings only cover the planes in flight (3 slots);
//     R, read as a stencil at p-1 and by its owner at p and p-2, keeps 6 slots.
//   - Every period is a divisor of 6: the R ring (6), the other rings and
//     barriers (3), the three-plane windows (3), the double-buffered stage planes
//     (2) and the d slots in tensor memory (6), and the barriers are
//     re-initialised for each work item so that their phases restart with it.
//     The z-march is laid out three ways (MODE): unrolled by 6, so that each
//     iteration's slots are constants; a plain loop whose slots (32-bit shared
//     addresses and absolute tensor-memory columns of this thread's cell) step by
//     constants in registers, the default, whose code fits the instruction cache;
//     or unrolled blocks of fast-path planes inside that loop.
//   - SPLIT variants replace the CTA barrier per plane by per-warp waits (below).
#include <type_traits>

#include "step_common.cuh"
#include "tmem_common.cuh"

namespace tdse {
namespace {

constexpr int kSlimU = 6;   // unroll of the z-march: every slot period divides it

template <class C>
struct SlimShape {
    typedef typename C::Real Real;
    static constexpr int H = C::H, PF = C::PF;
    static constexpr int NRS = 6;                      // R ring
    static constexpr int NBS = PF + 1;                 // I, cI, cR, d rings and barriers
    static constexpr int NSB = 2 * (H - 1);            // stage planes, double-buffered
    static constexpr int NPL = NRS + NBS * (C::KAHAN ? 4 : 2) + NSB;
    static constexpr size_t SMEM = static_cast<size_t>(NPL) * C::PLANE_BYTES + 8 * NBS + 128;
    static constexpr uint32_t TX_BYTES = C::PLANE_BYTES * (C::KAHAN ? 5 : 3);
    // tensor memory: the three-plane windows of F_1 .. F_{H-1} and 6 d slots
    static constexpr int NF = H - 1, NCMP = C::KAHAN ? 2 : 1, SLOT = C::VEC;
    static constexpr int NDT = 6;
    static constexpr int PHASE_COLS = NF * NCMP * SLOT;
    static constexpr int WIN_COLS = 3 * PHASE_COLS;
    static constexpr int THREAD_COLS = WIN_COLS + NDT * SLOT;
    static constexpr int NW = C::NT / 32;
    static constexpr int QUAD_COLS = ((NW + 3) / 4) * THREAD_COLS;
    static constexpr uint32_t NCOLS = tmem_cols_for(QUAD_COLS);
    static constexpr int MAX_RESIDENT_SMEM = 233472 / static_cast<int>(SMEM + 1024);
    static constexpr int MAX_RESIDENT_THREADS = 2048 / C::NT;
    static constexpr int MAX_RESIDENT = MAX_RESIDENT_SMEM < MAX_RESIDENT_THREADS ? MAX_RESIDENT_SMEM
                                                                                 : MAX_RESIDENT_THREADS;
    static_assert(sizeof(Real) == 4 && C::RPT == 1 && C::DSTASH, "FP32 fields, one row per thread");
    static_assert(H + 1 <= NDT, "d is read H planes back");
    static_assert(NRS >= PF + 3, "R is read two planes back");
    static constexpr bool UNROLLABLE = kSlimU % NRS == 0 && kSlimU % NBS == 0 && kSlimU % 3 == 0 &&
                                       kSlimU % 2 == 0 && kSlimU % NDT == 0;
    static_assert(QUAD_COLS <= 512, "windows exceed tensor memory");
    static_assert(MAX_RESIDENT * NCOLS <= 512, "co-resident CTAs exceed tensor memory");
    static_assert(C::MINB * (SMEM + 1024) <= 233472, "CTAs per SM exceed the shared memory");
};

// Slots of one iteration (it = it0 + k, it0 a multiple of kSlimU), as this thread
// uses them: shared-memory addresses of its own cell in the rings and absolute
// tensor-memory addresses of its columns, so that each access adds at most a
// constant (folded into the instruction).  Ring layout from the first R slot, in
// planes: R 0..5, I 6..8, d 9..11, then (Kahan) cI 12..14, cR 15..17, then the
// stage planes.
template <class C>
struct SlimSlots {
    typedef SlimShape<C> SS;
    static constexpr int PLANE = C::PLANE, NRS = SS::NRS, NBS = SS::NBS, NDT = SS::NDT, H = C::H;
    static constexpr uint32_t PB = 4u * PLANE;                    // bytes per plane
    static constexpr uint32_t OFF_I = NRS * PB, OFF_D = OFF_I + NBS * PB;
    static constexpr uint32_t OFF_CI = OFF_D + NBS * PB, OFF_CR = OFF_CI + NBS * PB;
    static constexpr uint32_t OFF_SB = (C::KAHAN ? OFF_CR + NBS * PB : OFF_CI);
    // from the I slot of a cell to the same cell of the other batch rings
    static constexpr uint32_t D_FROM_I = OFF_D - OFF_I, CI_FROM_I = OFF_CI - OFF_I, CR_FROM_I = OFF_CR - OFF_I;
    uint32_t r0, r1, r2;     // R at p, p-1, p-2
    uint32_t bb;             // I at p-1 (cI, cR and d at fixed distances)
    uint32_t sbp, sbc;       // stage planes read (previous iteration) and written
    uint32_t w0, w1, w2;     // window planes: old, center, new
    uint32_t d[H + 1];       // d at planes p, p-1, ..., p-H
    uint32_t rend, bend;     // ends of the rings (the thread's cell one past the last slot)
    uint32_t dbeg, dend;     // first and one past the last d slot
    int bar;                 // barrier slot
    uint32_t par;            // its phase parity
    // ring: shared address of the first R slot; own: the thread's cell in a plane
    __device__ __forceinline__ static SlimSlots at(int k, uint32_t tbase, uint32_t ring, int own)
    {
        SlimSlots x;
        const uint32_t cell = ring + 4u * static_cast<uint32_t>(own);
        x.r0 = cell + (k % NRS) * PB;
        x.r1 = cell + ((k + NRS - 1) % NRS) * PB;
        x.r2 = cell + ((k + NRS - 2) % NRS) * PB;
        x.bb = cell + OFF_I + (k % NBS) * PB;
        x.sbp = cell + OFF_SB + ((k + 1) & 1) * PB;
        x.sbc = cell + OFF_SB + (k & 1) * PB;
        x.w0 = tbase + static_cast<uint32_t>((k % 3) * SS::PHASE_COLS);
        x.w1 = tbase + static_cast<uint32_t>(((k + 1) % 3) * SS::PHASE_COLS);
        x.w2 = tbase + static_cast<uint32_t>(((k + 2) % 3) * SS::PHASE_COLS);
#pragma unroll
        for (int j = 0; j <= H; ++j)
            x.d[j] = tbase + static_cast<uint32_t>(SS::WIN_COLS + ((k - j + 2 * NDT) % NDT) * SS::SLOT);
        x.rend = cell + NRS * PB;
        x.bend = cell + OFF_I + NBS * PB;
        x.dbeg = tbase + SS::WIN_COLS;
        x.dend = tbase + SS::WIN_COLS + NDT * SS::SLOT;
        x.bar = k % NBS;
        x.par = static_cast<uint32_t>((k / NBS) & 1);
        return x;
    }
    // the next iteration's slots
    __device__ __forceinline__ void advance()
    {
        r2 = r1;
        r1 = r0;
        r0 += PB;
        if (r0 == rend) r0 -= NRS * PB;
        bb += PB;
        if (bb == bend) bb -= NBS * PB;
        const uint32_t t = sbp;
        sbp = sbc;
        sbc = t;
        const uint32_t w = w0;
        w0 = w1;
        w1 = w2;
        w2 = w;
#pragma unroll
        for (int j = H; j > 0; --j) d[j] = d[j - 1];
        d[0] += SS::SLOT;
        if (d[0] == dend) d[0] = dbeg;
        if (++bar == NBS) {
            bar = 0;
            par ^= 1u;
        }
    }
};

// Shared-memory accesses at a 32-bit shared address (plus a constant).
__device__ __forceinline__ float lds1(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void lds4(uint32_t a, float (&v)[4])
{
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3])
                 : "r"(a)
                 : "memory");
}
__device__ __forceinline__ void sts4(uint32_t a, const float (&v)[4])
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3])
                 : "memory");
}

// MODE: how the z-march is laid out.
//   kSlimUnrolled  unrolled by 6 with constant offsets: fewest instructions, but twelve
//                  copies of the stages (fast and general path) for the instruction cache;
//   kSlimRolled    a plain loop whose slot offsets rotate in registers: compact code;
//   kSlimHybrid    blocks of 6 planes that all take the fast path run unrolled (six
//                  copies of the fast stages), every other block the rolled loop.
constexpr int kSlimUnrolled = 0, kSlimRolled = 1, kSlimHybrid = 2;
// SPLIT: the CTA barrier per plane is split.  Each warp waits for its plane's loads
// itself, runs stage 1 (which reads only the loaded rings and its own tensor
// memory), then waits on an mbarrier that every warp arrives on when it finishes a
// plane; only then does it publish stage 1's row to the stage plane and run the
// stages that read the other warps' rows.  The loading thread refills a ring slot
// after that same wait.  So a warp's stage 1 overlaps the other warps' last stages.
template <class C, int MODE, bool SPLIT = false>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fused_step_slim_kernel(const MemberDev *__restrict__ members, const WorkDev *__restrict__ work,
                           int *counter, int *status, int in_buf, unsigned long long wait_ns)
{
    typedef float Real;
    typedef SlimShape<C> SS;
    typedef SlimSlots<C> Slots;
    static_assert(MODE == kSlimRolled || SS::UNROLLABLE, "every slot period must divide the unroll");
    constexpr int H = C::H, VEC = C::VEC, W = C::W, ROWS = C::ROWS, PLANE = C::PLANE;
    constexpr int PF = C::PF, NRS = SS::NRS, NBS = SS::NBS;
    constexpr bool KAHAN = C::KAHAN;

    extern __shared__ unsigned char smem_raw[];
    Real *ringR = reinterpret_cast<Real *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    Real *ringI = ringR + NRS * PLANE;
    Real *ringD = ringI + NBS * PLANE;
    Real *ringCI = ringD + NBS * PLANE;                 // Kahan only
    Real *ringCR = ringCI + (KAHAN ? NBS : 0) * PLANE;   // Kahan only
    Real *sbuf = ringCR + (KAHAN ? NBS : 0) * PLANE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbuf + SS::NSB * PLANE);
    const uint32_t uring = smem_u32(ringR);
    static_assert(Slots::OFF_SB == static_cast<uint32_t>(4 * (NRS + NBS * (KAHAN ? 4 : 2)) * PLANE),
                  "the slot layout follows the ring layout");
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ uint64_t s_done;   // SPLIT: every warp has finished the plane
    __shared__ uint32_t s_tmem;
    __shared__ ItemScalars S;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int qx = tid % C::TPX;
    const int r0 = tid / C::TPX;                         // this thread's region row
    // region rows of this warp (a row may continue in the neighbouring warp when
    // the threads of a row do not divide 32)
    const int warp_row0 = (warp * 32) / C::TPX, warp_row1 = (warp * 32 + 31) / C::TPX;
    // stages this warp runs: its rows leave the cone of stage s for s > smax_w
    const int smax_w = min(warp_row1, ROWS - 1 - warp_row0);
    // lanes whose x neighbour in the row sits in another warp: they read it from
    // the shared plane that holds the stage's input row
    const int lane = tid & 31;
    const bool x_from_smem_l = !C::ROW_IN_WARP && lane == 0 && qx > 0;
    const bool x_from_smem_r = !C::ROW_IN_WARP && lane == 31 && qx < C::TPX - 1;
    const int own = r0 * W + qx * VEC;
    const int off_ym = (r0 > 0 ? r0 - 1 : r0) * W + qx * VEC;
    const int off_yp = (r0 + 1 < ROWS ? r0 + 1 : r0) * W + qx * VEC;
    const int dym = off_ym - own, dyp = off_yp - own;   // the neighbouring rows' cells, from own

    if (warp == 0) tmem_alloc(&s_tmem, SS::NCOLS);
    if (tid == 0) {
        s_abort = 0;
        for (int b = 0; b < NBS; ++b) mbar_init(&bars[b], 1);
        if constexpr (SPLIT) mbar_init(&s_done, C::NT / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = s_tmem + ((static_cast<uint32_t>(warp & 3) * 32u) << 16) +
                           static_cast<uint32_t>(warp >> 2) * SS::THREAD_COLS;
    // column of field f (F_{f+1}), value (0) or compensation (1), within a window plane
    auto fcol = [](int f, int cmp) { return static_cast<uint32_t>((f * SS::NCMP + cmp) * SS::SLOT); };

    bool first_item = true;
    for (;;) {
        if (tid == 0) fetch_item(members, work, counter, in_buf, &s_item, S);
        __syncthreads();
        const int item = s_item;
        if (item >= work->total) break;
        const MemberDev &M = members[S.m];   // tensor maps only (thread 0)
        const int tile_x = S.tile_x, tile_y = S.tile_y, kz0 = S.kz0, kz1 = S.kz1;
        const int L0 = kz0 - H;
        const int nit = (kz1 - kz0) + 2 * H;
        const int G = S.G, nx = S.nx, ny = S.ny, nz = S.nz;
        const int bx = G + tile_x * C::TX - C::HX;
        const int by = G + tile_y * C::TY - H;
        const int xs = tile_x * C::TX - C::HX + qx * VEC;
        const int ys0 = tile_y * C::TY - H + r0;
        const bool zper = S.per_z != 0;
        const int mlo = S.mask_lo, mhi = nz - S.mask_hi;
        const float cxs = static_cast<float>(S.cx), cys = static_cast<float>(S.cy),
                    czs = static_cast<float>(S.cz);
        const float2 cx2 = make_float2(cxs, cxs), cy2 = make_float2(cys, cys),
                     cz2 = make_float2(czs, czs);
        const Real *maskz = reinterpret_cast<const Real *>(S.mask);
        const int kd = S.det_k;
        const bool flux_owner = kd >= kz0 && kd < kz1;

        auto inside = [&](int v) {
            return (S.per_x || (xs + v >= 0 && xs + v < nx)) && (S.per_y || (ys0 >= 0 && ys0 < ny));
        };
        bool walls = false;
#pragma unroll
        for (int v = 0; v < VEC; ++v) walls |= !inside(v);
        const bool store_row = qx * VEC >= C::HX && qx * VEC < C::HX + C::TX && xs < nx &&
                               r0 >= H && r0 < H + C::TY && ys0 < ny;
        const long long pitch = S.pitch;
        const bool seam = (S.per_x && (xs < G || xs >= nx - G)) || (S.per_y && (ys0 < G || ys0 >= ny - G));
        Real *outR = reinterpret_cast<Real *>(S.outR);
        Real *outI = reinterpret_cast<Real *>(S.outI);
        Real *outCR = reinterpret_cast<Real *>(S.outCR);
        Real *outCI = reinterpret_cast<Real *>(S.outCI);
        const long long out0 = static_cast<long long>(ys0 + G) * pitch + (xs + G);

        // windows start at zero (planes before the first computed one)
        {
            float zero[4] = {0.f, 0.f, 0.f, 0.f};
            for (int k = 0; k < 3; ++k)
                for (int f = 0; f < SS::NF; ++f)
                    for (int cmp = 0; cmp < SS::NCMP; ++cmp)
                        tmem_st4(tbase + static_cast<uint32_t>(k * SS::PHASE_COLS) + fcol(f, cmp), zero);
            tmem_wait_st();
        }
        // barriers restart their phases with each item (every load of the previous
        // item has been waited for)
        if (tid == 0) {
            if (!first_item) {
                for (int b = 0; b < NBS; ++b) {
                    mbar_inval(&bars[b]);
                    mbar_init(&bars[b], 1);
                }
                if constexpr (SPLIT) {
                    mbar_inval(&s_done);
                    mbar_init(&s_done, C::NT / 32);
                }
            }
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        first_item = false;
        const bool tile_walls = __syncthreads_or(walls) != 0;
        const int fast_lo = mlo + H;
        const int fast_hi = zper ? mhi + 1 : min(mhi + 1, nz);
        auto zwrap = [&](int L) { return zper ? ((L % nz) + nz) % nz : L; };

        // loads completing on barrier j % NBS: R and d at plane L0 + j, I and cI at
        // L0 + j - 1, cR at L0 + j - 2 (beyond a wall TMA fills zeros)
        auto issue = [&](int j) {
            const int L = L0 + j;
            uint64_t *bar = &bars[j % NBS];
            mbar_arrive_expect_tx(bar, SS::TX_BYTES);
            auto load = [&](Real *dst, const CUtensorMap *map, int z) { tma_load_3d(dst, map, bx, by, z, bar); };
            load(ringR + (j % NRS) * PLANE, &M.tm_R[in_buf], zwrap(L));
            load(ringD + (j % NBS) * PLANE, &M.tm_d, zwrap(L));
            load(ringI + (j % NBS) * PLANE, &M.tm_I[in_buf], zwrap(L - 1));
            if constexpr (KAHAN) {
                load(ringCI + (j % NBS) * PLANE, &M.tm_cI[in_buf], zwrap(L - 1));
                load(ringCR + (j % NBS) * PLANE, &M.tm_cR[in_buf], zwrap(L - 2));
            }
        };
        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int j = 0; j < PF && j < nit; ++j) issue(j);
        }
        int issued = min(PF, nit);
        int waited = 0;

        // The stages of iteration it (plane p) with its slots.
        // stage-to-stage registers (kept across the two halves of a split plane)
        Real zmh[VEC];    // z- neighbour of the previous stage = accumulator of this one
        Real prev[VEC];   // the previous stage's output: this stage's z+ neighbour
        Real held[VEC];   // SPLIT: stage 1's row, published after the plane barrier
        bool has_held = false;
        auto stages = [&](const int it, const int p, const Slots &sl, auto FASTc, auto SLOc, auto SHIc) {
            constexpr bool FAST = decltype(FASTc)::value;
            constexpr int SLO = decltype(SLOc)::value, SHI = decltype(SHIc)::value;
            // neighbouring rows of the stage planes read (previous iteration)
            const uint32_t sb_ym = sl.sbp + 4u * dym, sb_yp = sl.sbp + 4u * dyp;
            const bool p_out = !FAST && !zper && (p < 0 || p >= nz);
#pragma unroll
            for (int s = SLO; s <= SHI; ++s) {
                if (!FAST && it < 2 * s) continue;   // pipeline filling
                if (s > smax_w) continue;            // rows outside the cone
                const int q = p - s;
                const bool odd = (s & 1) != 0;
                bool q_out = false, absorb = false;
                Real mq = 1.f;
                if constexpr (!FAST) {
                    q_out = !zper && (q < 0 || q >= nz);
                    int qm = q;
                    if (zper) {
                        qm = q % nz;
                        if (qm < 0) qm += nz;
                    }
                    absorb = !q_out && (qm < mlo || qm >= mhi);
                    if (absorb) mq = maskz[qm];
                }
                Real zm[VEC], c[VEC], zp[VEC], ym[VEC], yp[VEC], dd[VEC], acc[VEC], cacc[VEC];
                tmem_ld4(sl.d[s], dd);   // d at plane q
                if (s == 1) {
                    lds4(sl.r2, zm);                           // R at p-2
                    lds4(sl.r1, c);                            // R at p-1
                    lds4(sl.r0, zp);                           // R at p
                    lds4(sl.bb, acc);                          // I at p-1
                    if constexpr (KAHAN) lds4(sl.bb + Slots::CI_FROM_I, cacc);   // cI at p-1
#pragma unroll
                    for (int v = 0; v < VEC; ++v)
                        if (p_out) zp[v] = 0.f;
                    lds4(sl.r1 + 4u * dym, ym);
                    lds4(sl.r1 + 4u * dyp, yp);
                    tmem_wait_ld();
                    after_wait(dd);
                } else {
                    tmem_ld4(sl.w0 + fcol(s - 2, 0), zm);
                    tmem_ld4(sl.w1 + fcol(s - 2, 0), c);
                    if (s >= 3 && KAHAN) tmem_ld4(sl.w0 + fcol(s - 3, 1), cacc);
                    lds4(sb_ym + (s - 2) * 2 * Slots::PB, ym);
                    lds4(sb_yp + (s - 2) * 2 * Slots::PB, yp);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        zp[v] = prev[v];
                        acc[v] = zmh[v];
                    }
                    if (s == 2 && KAHAN) lds4(sl.bb + Slots::CR_FROM_I, cacc);   // cR at p-2
                    tmem_wait_ld();
                    after_wait(dd);
                    after_wait(zm);
                    after_wait(c);
                    if (s >= 3 && KAHAN) after_wait(cacc);
                }
                if (s >= 3 && odd && absorb) {   // I of the previous step carries its absorbing factor
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        acc[v] = mul_rn(acc[v], mq);
                        if constexpr (KAHAN) cacc[v] = mul_rn(cacc[v], mq);
                    }
                }

                Real out[VEC], cout[VEC];
                {
                    Real xl = __shfl_up_sync(kFull, c[VEC - 1], 1);
                    Real xr = __shfl_down_sync(kFull, c[0], 1);
                    if constexpr (!C::ROW_IN_WARP) {
                        // the stage's input row: R at p-1 in its ring (stage 1), else the
                        // stage plane of F_{s-1} written in the previous iteration
                        const uint32_t crow = s == 1 ? sl.r1 : sl.sbp + (s - 2) * 2 * Slots::PB;
                        if (x_from_smem_l) xl = lds1(crow - 4u);
                        if (x_from_smem_r) xr = lds1(crow + 4u * VEC);
                    }
                    update_row_f32<KAHAN, VEC>(odd, c, xl, xr, ym, yp, zm, zp, dd, acc, cacc, cx2, cy2,
                                               cz2, out, cout);
                }
                if (!odd && absorb) {   // Eq. 8 step complete: absorbing factor on R
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        out[v] = mul_rn(out[v], mq);
                        if constexpr (KAHAN) cout[v] = mul_rn(cout[v], mq);
                    }
                }
                if constexpr (!FAST) {
                    if (walls || q_out) {
                        const Real zq = q_out ? 0.f : 1.f;
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            const Real keep = inside(v) ? 1.f : 0.f;
                            out[v] *= keep * zq;
                            if constexpr (KAHAN) cout[v] *= keep * zq;
                        }
                    }
                    // detector flux of step (s+1)/2: R^n at planes kd, kd+1 and the new I
                    if (odd && s < H && flux_owner && q == kd + 1) {
                        Real ilo[VEC];   // I at plane kd: the center of stage s's window
                        tmem_ld4(sl.w1 + fcol(s - 1, 0), ilo);
                        tmem_wait_ld();
                        after_wait(ilo);
                        if (store_row) {
                            const int pix = ys0 * nx + xs;
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                const double j = S.cj * (static_cast<double>(zm[v]) * out[v] -
                                                         static_cast<double>(c[v]) * ilo[v]);
                                S.flux[pix + v] += j * S.dt;
                                if (s == H - 1) S.jlast[pix + v] = j;
                            }
                        }
                    }
                }

                if (s < H) {
                    tmem_st4(sl.w2 + fcol(s - 1, 0), out);
                    if constexpr (KAHAN) tmem_st4(sl.w2 + fcol(s - 1, 1), cout);
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        prev[v] = out[v];
                        zmh[v] = zm[v];
                    }
                    if (SPLIT && s == 1) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) held[v] = out[v];
                        has_held = true;
                    } else {
                        sts4(sl.sbc + (s - 1) * 2 * Slots::PB, out);
                    }
                } else {
                    // I of the last step: the center of F_{H-1}'s window
                    Real vi[VEC], vci[VEC];
                    tmem_ld4(sl.w1 + fcol(H - 2, 0), vi);
                    if constexpr (KAHAN) tmem_ld4(sl.w1 + fcol(H - 2, 1), vci);
                    tmem_wait_ld();
                    after_wait(vi);
                    if constexpr (KAHAN) after_wait(vci);
                    if (store_row && (FAST || (q >= kz0 && q < kz1))) {
                        if (absorb) {
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                vi[v] = mul_rn(vi[v], mq);
                                if constexpr (KAHAN) vci[v] = mul_rn(vci[v], mq);
                            }
                        }
                        const long long zoff = static_cast<long long>(q) * S.plane;
                        store_output_row<Real, KAHAN, VEC>(S, outR, outI, outCR, outCI, zoff + out0, pitch,
                                                           seam, xs, ys0, out, vi, cout, vci);
                    }
                }
            }
        };

        // the stages SLO..SHI of plane p (ONLY_FAST: the caller knows the plane takes the fast path)
        auto run_stages = [&](const int it, const int p, const Slots &sl, auto ONLY_FASTc, auto SLOc, auto SHIc) {
            if constexpr (decltype(ONLY_FASTc)::value) {
                stages(it, p, sl, std::true_type{}, SLOc, SHIc);
            } else {
                const bool fast = !tile_walls && it >= 2 * H && p >= fast_lo && p < fast_hi &&
                                  !(flux_owner && p >= kd + 2 && p <= kd + H);
                if (fast)
                    stages(it, p, sl, std::true_type{}, SLOc, SHIc);
                else
                    stages(it, p, sl, std::false_type{}, SLOc, SHIc);
            }
        };
        typedef std::integral_constant<int, 1> S1;
        typedef std::integral_constant<int, 2> S2;
        typedef std::integral_constant<int, H> SH;
        // a bounded wait taken by a whole warp: it goes on only if every lane saw the
        // phase complete; an expired wait raises the abort flag
        auto warp_wait = [&](uint64_t *bar, uint32_t parity) -> bool {
            const int r = __reduce_min_sync(kFull, mbar_wait_or_abort(bar, parity, wait_ns, &s_abort));
            if (r == 0) {
                atomicOr(status, 1);
                s_abort = 1;
            }
            return r == 1;
        };

        // One iteration: wait for plane L0 + it, refill, d to tensor memory, stages.
        auto plane_step = [&](const int it, const Slots &sl, auto ONLY_FASTc) -> bool {
            const int p = L0 + it;
            if constexpr (!SPLIT) {
                if (tid == 0) {
                    if (mbar_wait_bounded(&bars[sl.bar], sl.par, wait_ns)) {
                        waited = it + 1;
                    } else {
                        atomicOr(status, 1);
                        s_abort = 1;
                    }
                }
                __syncthreads();   // plane p has landed; the previous iteration's reads are done
                if (s_abort) return false;
                if (it + PF < nit) {
                    if (tid == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(it + PF);
                    }
                    issued = it + PF + 1;
                }
                tmem_wait_st();   // the previous iteration's window planes are in TMEM
                {
                    Real dp[VEC];
                    lds4(sl.bb + Slots::D_FROM_I, dp);
                    tmem_st4(sl.d[0], dp);
                }
                run_stages(it, p, sl, ONLY_FASTc, S1{}, SH{});
                return true;
            } else {
                if (!warp_wait(&bars[sl.bar], sl.par)) return false;   // plane p has landed
                if (tid == 0) waited = it + 1;
                tmem_wait_st();
                {
                    Real dp[VEC];
                    lds4(sl.bb + Slots::D_FROM_I, dp);
                    tmem_st4(sl.d[0], dp);
                }
                has_held = false;
                run_stages(it, p, sl, ONLY_FASTc, S1{}, S1{});
                // every warp has finished plane p - 1: its stage rows are readable, and
                // the slots it read (the stage plane written next, the ring slot refilled
                // next) are free
                if (it > 0 && !warp_wait(&s_done, static_cast<uint32_t>((it - 1) & 1))) return false;
                if (it + PF < nit) {
                    if (tid == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(it + PF);
                    }
                    issued = it + PF + 1;
                }
                if (has_held) sts4(sl.sbc, held);
                run_stages(it, p, sl, ONLY_FASTc, S2{}, SH{});
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&s_done);
                return true;
            }
        };
        const std::false_type any{};
        const std::true_type only_fast{};

        if constexpr (MODE == kSlimRolled) {
            Slots sl = Slots::at(0, tbase, uring, own);
            for (int it = 0; it < nit; ++it) {
                if (!plane_step(it, sl, any)) break;
                sl.advance();
            }
        } else if constexpr (MODE == kSlimUnrolled) {
            for (int it0 = 0; it0 < nit; it0 += kSlimU) {
                if (!plane_step(it0, Slots::at(0, tbase, uring, own), any)) break;
                if (it0 + 1 >= nit || !plane_step(it0 + 1, Slots::at(1, tbase, uring, own), any)) break;
                if (it0 + 2 >= nit || !plane_step(it0 + 2, Slots::at(2, tbase, uring, own), any)) break;
                if (it0 + 3 >= nit || !plane_step(it0 + 3, Slots::at(3, tbase, uring, own), any)) break;
                if (it0 + 4 >= nit || !plane_step(it0 + 4, Slots::at(4, tbase, uring, own), any)) break;
                if (it0 + 5 >= nit || !plane_step(it0 + 5, Slots::at(5, tbase, uring, own), any)) break;
            }
        } else {
            bool ok = true;
            for (int it0 = 0; it0 < nit && ok; it0 += kSlimU) {
                const int p0 = L0 + it0;
                const bool block_fast = !tile_walls && it0 >= 2 * H && it0 + kSlimU <= nit && p0 >= fast_lo &&
                                        p0 + kSlimU - 1 < fast_hi &&
                                        !(flux_owner && p0 <= kd + H && p0 + kSlimU - 1 >= kd + 2);
                if (block_fast) {
                    ok = plane_step(it0, Slots::at(0, tbase, uring, own), only_fast) && plane_step(it0 + 1, Slots::at(1, tbase, uring, own), only_fast) &&
                         plane_step(it0 + 2, Slots::at(2, tbase, uring, own), only_fast) &&
                         plane_step(it0 + 3, Slots::at(3, tbase, uring, own), only_fast) &&
                         plane_step(it0 + 4, Slots::at(4, tbase, uring, own), only_fast) && plane_step(it0 + 5, Slots::at(5, tbase, uring, own), only_fast);
                } else {
                    Slots sl = Slots::at(0, tbase, uring, own);
                    for (int k = 0; k < kSlimU && it0 + k < nit && ok; ++k) {
                        ok = plane_step(it0 + k, sl, any);
                        sl.advance();
                    }
                }
            }
        }

        __syncthreads();   // every thread has left the z-march: all read the same s_abort
        if (s_abort) {
            // wait (bounded) for the loads still in flight, then leave (freeing TMEM below)
            if (tid == 0) {
                for (int l = waited; l < issued; ++l)
                    if (!mbar_wait_bounded(&bars[l % NBS], static_cast<uint32_t>((l / NBS) & 1)))
                        atomicOr(status, 4);   // the CTA leaves with a load still in flight
            }
            __syncthreads();
            break;
        }
        tmem_wait_st();
        __syncthreads();
    }

    tmem_wait_st();
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(s_tmem, SS::NCOLS);
}

template <class C, int MODE, bool SPLIT>
cudaError_t launch_slim_cfg(const StepLaunch &L)
{
    typedef SlimShape<C> SS;
    static std::atomic<uint64_t> smem_allowed{0};   // one bit per device
    cudaError_t e = allow_dynamic_smem(fused_step_slim_kernel<C, MODE, SPLIT>, SS::SMEM, smem_allowed);
    if (e != cudaSuccess) return e;
    fused_step_slim_kernel<C, MODE, SPLIT><<<L.grid, C::NT, SS::SMEM, L.stream>>>(
        L.members, L.work, L.counter, L.status, L.in_buf, L.wait_ns);
    return cudaGetLastError();
}

template <class C>
void fill_slim_config(StepConfig *cfg)
{
    cfg->tile_x = C::TX;
    cfg->tile_y = C::TY;
    cfg->box_x = C::W;
    cfg->box_y = C::ROWS;
    cfg->threads = C::NT;
    cfg->smem = SlimShape<C>::SMEM;
    cfg->ctas_per_sm = C::MINB;
}

}  // namespace

#define TDSE_SLIM_VARIANT_S(FN, MODE, SPLIT, ...)                                        \
    cudaError_t launch_##FN(const StepLaunch &L) { return launch_slim_cfg<Cfg<__VA_ARGS__>, MODE, SPLIT>(L); } \
    void fill_##FN(StepConfig *cfg) { fill_slim_config<Cfg<__VA_ARGS__>>(cfg); }
#define TDSE_SLIM_VARIANT(FN, MODE, ...) TDSE_SLIM_VARIANT_S(FN, MODE, false, __VA_ARGS__)

// Cfg<Real, 2T, threads per row, rows, rows per thread, Kahan, planes prefetched, CTAs per SM,
//     d kept in TMEM, own rings>; "slim": unrolled, "roll": rolled, "hyb": hybrid (MODE)
TDSE_SLIM_VARIANT(slim_k32_t2_w32_r32x1_pf2_b2, kSlimUnrolled, float, 4, 8, 32, 1, true, 2, 2, true, true)
TDSE_SLIM_VARIANT(roll_k32_t2_w32_r32x1_pf2_b2, kSlimRolled, float, 4, 8, 32, 1, true, 2, 2, true, true)
TDSE_SLIM_VARIANT_S(split_k32_t2_w32_r32x1_pf2_b2, kSlimRolled, true, float, 4, 8, 32, 1, true, 2, 2, true, true)
TDSE_SLIM_VARIANT_S(split_f32_t2_w32_r32x1_pf2_b2, kSlimRolled, true, float, 4, 8, 32, 1, false, 2, 2, true, true)
TDSE_SLIM_VARIANT(roll_k32_t2_w32_r28x1_pf2_b2, kSlimRolled, float, 4, 8, 28, 1, true, 2, 2, true, true)
TDSE_SLIM_VARIANT(roll_f32_t2_w32_r32x1_pf2_b2, kSlimRolled, float, 4, 8, 32, 1, false, 2, 2, true, true)
TDSE_SLIM_VARIANT(roll_k32_t2_w32_r32x1_pf3_b2, kSlimRolled, float, 4, 8, 32, 1, true, 3, 2, true, true)
TDSE_SLIM_VARIANT(roll_k32_t2_r32x1_pf2, kSlimRolled, float, 4, 16, 32, 1, true, 2, 1, true, true)
TDSE_SLIM_VARIANT(roll_k32_t2_r32x1_pf3, kSlimRolled, float, 4, 16, 32, 1, true, 3, 1, true, true)
TDSE_SLIM_VARIANT_S(split_k32_t2_r32x1_pf2, kSlimRolled, true, float, 4, 16, 32, 1, true, 2, 1, true, true)
TDSE_SLIM_VARIANT_S(split_k32_t2_r32x1_pf3, kSlimRolled, true, float, 4, 16, 32, 1, true, 3, 1, true, true)
TDSE_SLIM_VARIANT_S(split_f32_t2_r32x1_pf2, kSlimRolled, true, float, 4, 16, 32, 1, false, 2, 1, true, true)
TDSE_SLIM_VARIANT_S(split_f32_t2_r32x1_pf3, kSlimRolled, true, float, 4, 16, 32, 1, false, 3, 1, true, true)
// 72 x 32 boxes (64 x 24 tiles): 18 threads per row, so rows continue across warps
TDSE_SLIM_VARIANT_S(split_k32_t2_w72_r32x1_pf2, kSlimRolled, true, float, 4, 18, 32, 1, true, 2, 1, true, true)
TDSE_SLIM_VARIANT_S(split_f32_t2_w72_r32x1_pf2, kSlimRolled, true, float, 4, 18, 32, 1, false, 2, 1, true, true)
TDSE_SLIM_VARIANT_S(split_f32_t2_w72_r32x1_pf3, kSlimRolled, true, float, 4, 18, 32, 1, false, 3, 1, true, true)
TDSE_SLIM_VARIANT(roll_f32_t2_w32_r32x1_pf3_b2, kSlimRolled, float, 4, 8, 32, 1, false, 3, 2, true, true)
TDSE_SLIM_VARIANT(roll_f32_t2_r32x1_pf3, kSlimRolled, float, 4, 16, 32, 1, false, 3, 1, true, true)
TDSE_SLIM_VARIANT(hyb_k32_t2_w32_r32x1_pf2_b2, kSlimHybrid, float, 4, 8, 32, 1, true, 2, 2, true, true)
TDSE_SLIM_VARIANT(hyb_f32_t2_w32_r32x1_pf2_b2, kSlimHybrid, float, 4, 8, 32, 1, false, 2, 2, true, true)

}  // namespace tdse
