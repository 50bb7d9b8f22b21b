// Fused leapfrog step with the stage windows in tensor memory (arXiv 2401.07416,
// Sec. 2.1, Eqs. 8-9), FP32 and FP32 + Kahan.
//
// Same schedule and arithmetic as fused_step_kernel: a CTA marches an xy tile
// along z and runs the 2T half-step stages of T fused time steps as a pipeline,
// stage s on plane p - s while plane p arrives by TMA.  The difference is where
// the three-plane windows (old q-1, center q, new q+1) of the intermediate
// fields F_1 .. F_{2T-1}, and of their Kahan compensation terms, are kept: in
// tensor memory (TMEM: 128 lanes x 512 columns of 32 bits per SM, beside the
// register file) instead of registers.  A window value is only ever read back
// by the thread that wrote it, which is TMEM's access pattern: warp w reaches
// lanes 32 (w mod 4) .. 32 (w mod 4) + 31, and warps sharing a lane quadrant use
// disjoint column ranges.  Registers then hold only one stage's temporaries, so
// a CTA runs one tile row per thread with twice the warps of the register-window
// kernel.  The phase of each window (which of its three slots is old, center,
// new) is a runtime column offset, so the z-march needs no unrolling.
//
// The newest plane of a window (the stage output just computed) is used by the
// next stage straight from registers; old and center planes come from TMEM
// (tcgen05.ld, then tcgen05.wait::ld).  Stores of new planes (tcgen05.st) are
// waited for once per iteration, before any load that could read them.
#include <type_traits>

#include "step_common.cuh"
#include "tmem_common.cuh"

namespace tdse {
namespace {

// TMEM footprint of a configuration.
template <class C>
struct TmemShape {
    static constexpr int NW = C::NT / 32;                    // warps
    static constexpr int NF = C::H - 1;                      // windowed fields F_1 .. F_{H-1}
    static constexpr int NCMP = C::KAHAN ? 2 : 1;            // value (and compensation)
    static constexpr int SLOT = C::RPT * C::VEC;             // columns of one window plane
    static constexpr int NDT = C::H + 2 <= 8 ? 8 : 16;      // d planes kept (p .. p-H), a power of two
    static constexpr int PHASE_COLS = NF * NCMP * SLOT;      // one window plane of every field
    static constexpr int WIN_COLS = 3 * PHASE_COLS;          // one thread's windows
    static constexpr int THREAD_COLS = WIN_COLS + NDT * SLOT;
    static constexpr int QUAD_COLS = ((NW + 3) / 4) * THREAD_COLS;   // warps w, w+4, ... share a quadrant
    static constexpr uint32_t NCOLS = tmem_cols_for(QUAD_COLS);
    static_assert(QUAD_COLS <= 512, "windows exceed tensor memory");
    // CTAs that shared memory and the thread limit let share an SM must fit in TMEM
    // together (an allocation that cannot be met would wait for another CTA to exit)
    static constexpr int MAX_RESIDENT_SMEM = 233472 / static_cast<int>(C::SMEM + 1024);
    static constexpr int MAX_RESIDENT_THREADS = 2048 / C::NT;
    static constexpr int MAX_RESIDENT = MAX_RESIDENT_SMEM < MAX_RESIDENT_THREADS ? MAX_RESIDENT_SMEM
                                                                                 : MAX_RESIDENT_THREADS;
    static_assert(MAX_RESIDENT * NCOLS <= 512, "co-resident CTAs exceed tensor memory");
    static_assert(sizeof(typename C::Real) == 4, "TMEM windows are for FP32 fields");
    static_assert(C::H >= 2, "at least one full step per launch");
    static_assert(C::DSTASH, "the tensor-memory kernel keeps d in TMEM");
};

// Synchronisation of the z-march, two forms (WS):
//   false  thread 0 waits for each plane's loads and refills the rings, and one
//          CTA barrier per plane orders everything;
//   true   a producer warp (after the C::NT compute threads) issues the loads; a
//          compute warp waits for its plane's loads (full[]) and for its two
//          neighbouring warps to finish the previous plane (nbr[], the only
//          shared-memory exchange between warps: the stage planes of the rows at
//          its edges), and reports each finished plane (done[]), after which the
//          producer may refill that plane's ring slots.  No CTA-wide barrier inside
//          the z-march: warps drift apart by up to the ring depth.
template <class C, bool WS>
struct TmemSync {
    static constexpr int NWC = C::NT / 32;                     // compute warps
    static constexpr int THREADS = C::NT + (WS ? 32 : 0);
    static constexpr size_t SMEM = C::SMEM + (WS ? 8u * (C::NB + 2 * NWC) : 0u);
    static_assert(!WS || NWC >= 2, "neighbour barriers need two compute warps");
    static_assert(!WS || C::MINB * (SMEM + 1024) <= 233472, "CTAs per SM exceed the shared memory");
    static_assert(!WS || C::PF >= 1, "the producer needs at least one plane ahead");
};

template <class C, bool WS>
__global__ void __launch_bounds__(TmemSync<C, WS>::THREADS, C::MINB)
    fused_step_tmem_kernel(const MemberDev *__restrict__ members, const WorkDev *__restrict__ work,
                           int *counter, int *status, int in_buf,
                           unsigned long long wait_ns)
{
    static_assert(C::ROW_IN_WARP, "x neighbours by shuffles need each region row inside one warp");
    typedef float Real;
    typedef TmemShape<C> TS;
    constexpr int H = C::H, VEC = C::VEC, W = C::W, ROWS = C::ROWS, PLANE = C::PLANE;
    constexpr int RPT = C::RPT, NB = C::NB, PF = C::PF, NR = C::NR, NI = C::NI, ND = C::ND;
    constexpr int SLOT = C::NFC * PLANE;    // one ring slot: a field (and its compensation)
    constexpr int OFF_C = PLANE;            // compensation term within a slot
    constexpr int NWC = TmemSync<C, WS>::NWC;

    extern __shared__ unsigned char smem_raw[];
    Real *ringA = reinterpret_cast<Real *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    Real *ringI = ringA + NR * SLOT;
    Real *ringD = ringI + NI * SLOT;
    Real *sbuf = ringD + ND * PLANE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbuf + C::NSB * PLANE);   // full[NB]
    uint64_t *done = bars + NB;          // WS: done[NB]
    uint64_t *nbr = done + NB;           // WS: nbr[NWC][2], by iteration parity
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ uint32_t s_tmem;
    __shared__ ItemScalars S;

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int lane = tid & 31;
    const bool producer = WS && warp == NWC;
    const volatile int *abort_flag = &s_abort;
    const int qx = tid % C::TPX;
    const int r0 = (tid / C::TPX) * RPT;                 // first region row of this thread
    const int warp_row0 = warp * C::RW;
    const int own = r0 * W + qx * VEC;                   // row r of this thread: own + r * W
    const int off_ym = (r0 > 0 ? r0 - 1 : r0) * W + qx * VEC;
    const int off_yp = (r0 + RPT < ROWS ? r0 + RPT : r0 + RPT - 1) * W + qx * VEC;

    if (warp == 0) tmem_alloc(&s_tmem, TS::NCOLS);
    if (tid == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
        if constexpr (WS) {
            for (int b = 0; b < NB; ++b) mbar_init(&done[b], NWC);
            for (int w = 0; w < NWC; ++w)
                for (int k = 0; k < 2; ++k) mbar_init(&nbr[2 * w + k], (w > 0) + (w < NWC - 1));
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    // this thread's lane and column range: lane quadrant warp % 4, column group warp / 4
    const uint32_t tbase = s_tmem + ((static_cast<uint32_t>(warp & 3) * 32u) << 16) +
                           static_cast<uint32_t>(warp >> 2) * TS::THREAD_COLS;
    // Column layout of a thread: window plane k (0..2) of every field first (k
    // outermost, so one base address per phase serves all fields), then the d ring.
    // Within a phase: field f (F_{f+1}), value (0) or compensation (1).
    auto fcol = [](int f, int cmp) { return static_cast<uint32_t>((f * TS::NCMP + cmp) * TS::SLOT); };
    auto pbase = [&](int k) { return tbase + static_cast<uint32_t>(k * TS::PHASE_COLS); };
    const uint32_t dbase = tbase + TS::WIN_COLS;
    auto dcol = [&](int j) { return dbase + static_cast<uint32_t>((j & (TS::NDT - 1)) * TS::SLOT); };

    long long gbase = 0;   // loads issued by this CTA before the current item

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

        auto inside = [&](int r, int v) {
            return (S.per_x || (xs + v >= 0 && xs + v < nx)) && (S.per_y || (ys0 + r >= 0 && ys0 + r < ny));
        };
        bool walls = false;
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int v = 0; v < VEC; ++v) walls |= !inside(r, v);
        walls = walls && !producer;
        const bool col_in = qx * VEC >= C::HX && qx * VEC < C::HX + C::TX && xs < nx;
        bool store_row[RPT];
        bool any_store = false;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            store_row[r] = col_in && r0 + r >= H && r0 + r < H + C::TY && ys0 + r < ny;
            any_store |= store_row[r];
        }
        const long long pitch = S.pitch;
        const bool seam = (S.per_x && (xs < G || xs >= nx - G)) ||
                          (S.per_y && (ys0 < G || ys0 + RPT - 1 >= ny - G));
        Real *outR = reinterpret_cast<Real *>(S.outR);
        Real *outI = reinterpret_cast<Real *>(S.outI);
        Real *outCR = reinterpret_cast<Real *>(S.outCR);
        Real *outCI = reinterpret_cast<Real *>(S.outCI);
        const long long out0 = static_cast<long long>(ys0 + G) * pitch + (xs + G);

        // Windows start at zero (planes before the first computed one), as in the
        // register-window kernel.
        if (!producer) {
            float zero[4] = {0.f, 0.f, 0.f, 0.f};
            for (int f = 0; f < TS::NF; ++f)
                for (int k = 0; k < 3; ++k)
                    for (int cmp = 0; cmp < TS::NCMP; ++cmp)
#pragma unroll
                        for (int r = 0; r < RPT; ++r) tmem_st4(pbase(k) + fcol(f, cmp) + r * VEC, zero);
            tmem_wait_st();
        }

        const bool tile_walls = __syncthreads_or(walls) != 0;
        const int fast_lo = mlo + H;
        const int fast_hi = zper ? mhi + 1 : min(mhi + 1, nz);

        int headA = 0, headI = 0, headD = 0;
        int headB = static_cast<int>(gbase % NB);
        uint32_t phase = static_cast<uint32_t>((gbase / NB) & 1);

        auto issue = [&](int l, int ahead) {
            const int L = L0 + l;
            const int zc = zper ? ((L % nz) + nz) % nz : L;
            int b = headB + ahead; if (b >= NB) b -= NB;
            int a = headA + ahead; if (a >= NR) a -= NR;
            int i = headI + ahead; if (i >= NI) i -= NI;
            int d = headD + ahead; if (d >= ND) d -= ND;
            uint64_t *bar = &bars[b];
            Real *slotR = ringA + a * SLOT;
            Real *slotI = ringI + i * SLOT;
            mbar_arrive_expect_tx(bar, C::TX_BYTES);
            tma_load_3d(slotR, &M.tm_R[in_buf], bx, by, zc, bar);
            tma_load_3d(slotI, &M.tm_I[in_buf], bx, by, zc, bar);
            if constexpr (C::KAHAN) {
                tma_load_3d(slotR + OFF_C, &M.tm_cR[in_buf], bx, by, zc, bar);
                tma_load_3d(slotI + OFF_C, &M.tm_cI[in_buf], bx, by, zc, bar);
            }
            tma_load_3d(ringD + d * PLANE, &M.tm_d, bx, by, zc, bar);
        };

        // The same loads for the producer warp: plane L0 + l into ring slots l mod NR,
        // NI, ND (the rings restart with each item) and barrier slot (gbase + l) mod NB.
        auto issue_at = [&](int l) {
            const int L = L0 + l;
            const int zc = zper ? ((L % nz) + nz) % nz : L;
            uint64_t *bar = &bars[(gbase + l) % NB];
            Real *slotR = ringA + (l % NR) * SLOT;
            Real *slotI = ringI + (l % NI) * SLOT;
            mbar_arrive_expect_tx(bar, C::TX_BYTES);
            tma_load_3d(slotR, &M.tm_R[in_buf], bx, by, zc, bar);
            tma_load_3d(slotI, &M.tm_I[in_buf], bx, by, zc, bar);
            if constexpr (C::KAHAN) {
                tma_load_3d(slotR + OFF_C, &M.tm_cR[in_buf], bx, by, zc, bar);
                tma_load_3d(slotI + OFF_C, &M.tm_cI[in_buf], bx, by, zc, bar);
            }
            tma_load_3d(ringD + (l % ND) * PLANE, &M.tm_d, bx, by, zc, bar);
        };

        if (!WS && tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int l = 0; l < PF && l < nit; ++l) issue(l, l);
        }
        int issued = WS ? 0 : min(PF, nit);
        int waited = 0;

        auto stages = [&](const int it, const int p, const uint32_t K0, const uint32_t K1, const uint32_t K2,
                          const int dj, const Real *A0, const Real *A1, const Real *A2,
                          const Real *I1, const Real *sb_prev, Real *sb_cur, auto FASTc) {
            constexpr bool FAST = decltype(FASTc)::value;
            const bool p_out = !FAST && !zper && (p < 0 || p >= nz);
            // The z- neighbour of stage s is F_{s-1} at plane p-s-1, which is also the
            // accumulator of stage s+1 (F_{s-1} at plane p-(s+1)): it stays in registers
            // from one stage to the next (for stage 1, R at plane p-2 from shared memory).
            // Stage s runs only when stage s-1 ran in the same iteration (the pipeline
            // fill and the cone both shrink with s), so zmh always holds that value.
            Real zmh[RPT][VEC];
            Real prev[RPT][VEC];   // the previous stage's output: this stage's z+ neighbour
#pragma unroll
            for (int s = 1; s <= H; ++s) {
                if (!FAST && it < 2 * s) continue;                            // pipeline filling
                if (warp_row0 + C::RW <= s || warp_row0 >= ROWS - s) continue;  // rows outside the cone
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

                Real zm[RPT][VEC], c[RPT][VEC], zp[RPT][VEC], ym[VEC], yp[VEC], dd[RPT][VEC];
                Real acc[RPT][VEC], cacc[RPT][VEC];
#pragma unroll
                for (int r = 0; r < RPT; ++r) tmem_ld4(dcol(dj - s) + r * VEC, dd[r]);   // d at plane q
                if (s == 1) {
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        ld_vec<Real>(A2 + own + r * W, zm[r]);
                        ld_vec<Real>(A1 + own + r * W, c[r]);
                        ld_vec<Real>(A0 + own + r * W, zp[r]);
                        ld_vec<Real>(I1 + own + r * W, acc[r]);
                        if constexpr (C::KAHAN) ld_vec<Real>(I1 + OFF_C + own + r * W, cacc[r]);
#pragma unroll
                        for (int v = 0; v < VEC; ++v)
                            if (p_out) zp[r][v] = 0.f;
                    }
                    ld_vec<Real>(A1 + off_ym, ym);
                    ld_vec<Real>(A1 + off_yp, yp);
                    tmem_wait_ld();
#pragma unroll
                    for (int r = 0; r < RPT; ++r) after_wait(dd[r]);
                } else {
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        tmem_ld4(K0 + fcol(s - 2, 0) + r * VEC, zm[r]);
                        tmem_ld4(K1 + fcol(s - 2, 0) + r * VEC, c[r]);
                        if (s >= 3 && C::KAHAN) tmem_ld4(K0 + fcol(s - 3, 1) + r * VEC, cacc[r]);
                    }
                    const Real *Sp = sb_prev + (s - 2) * 2 * PLANE;
                    ld_vec<Real>(Sp + off_ym, ym);
                    ld_vec<Real>(Sp + off_yp, yp);
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            zp[r][v] = prev[r][v];
                            acc[r][v] = zmh[r][v];
                        }
                        if (s == 2 && C::KAHAN) ld_vec<Real>(A2 + OFF_C + own + r * W, cacc[r]);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        after_wait(dd[r]);
                        after_wait(zm[r]);
                        after_wait(c[r]);
                        if (s >= 3 && C::KAHAN) after_wait(cacc[r]);
                    }
                }
                if (s >= 3 && odd && absorb) {   // I of the previous step carries its absorbing factor
#pragma unroll
                    for (int r = 0; r < RPT; ++r)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            acc[r][v] = mul_rn(acc[r][v], mq);
                            if constexpr (C::KAHAN) cacc[r][v] = mul_rn(cacc[r][v], mq);
                        }
                }

                Real out[RPT][VEC], cout[RPT][VEC];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const Real xl = __shfl_up_sync(kFull, c[r][VEC - 1], 1);
                    const Real xr = __shfl_down_sync(kFull, c[r][0], 1);
                    update_row_f32<C::KAHAN, VEC>(odd, c[r], xl, xr, r == 0 ? ym : c[r - 1],
                                                  r == RPT - 1 ? yp : c[r + 1], zm[r], zp[r], dd[r],
                                                  acc[r], cacc[r], cx2, cy2, cz2, out[r], cout[r]);
                }
                if (!odd && absorb) {   // Eq. 8 step complete: absorbing factor on R
#pragma unroll
                    for (int r = 0; r < RPT; ++r)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            out[r][v] = mul_rn(out[r][v], mq);
                            if constexpr (C::KAHAN) cout[r][v] = mul_rn(cout[r][v], mq);
                        }
                }
                if constexpr (!FAST) {
                    if (walls || q_out) {
                        const Real zq = q_out ? 0.f : 1.f;
#pragma unroll
                        for (int r = 0; r < RPT; ++r)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                const Real keep = inside(r, v) ? 1.f : 0.f;
                                out[r][v] *= keep * zq;
                                if constexpr (C::KAHAN) cout[r][v] *= keep * zq;
                            }
                    }

                    // detector flux of step (s+1)/2: R^n at planes kd, kd+1 and the new I
                    if (odd && s < H && flux_owner && q == kd + 1) {
                        Real ilo[RPT][VEC];   // I at plane kd: the previous output of stage s
#pragma unroll
                        for (int r = 0; r < RPT; ++r) tmem_ld4(K1 + fcol(s - 1, 0) + r * VEC, ilo[r]);
                        tmem_wait_ld();
#pragma unroll
                        for (int r = 0; r < RPT; ++r) after_wait(ilo[r]);
                        if (any_store) {
#pragma unroll
                            for (int r = 0; r < RPT; ++r) {
                                if (!store_row[r]) continue;
                                const int pix = (ys0 + r) * nx + xs;
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    const double j = S.cj * (static_cast<double>(zm[r][v]) * out[r][v] -
                                                             static_cast<double>(c[r][v]) * ilo[r][v]);
                                    S.flux[pix + v] += j * S.dt;
                                    if (s == H - 1) S.jlast[pix + v] = j;
                                }
                            }
                        }
                    }
                }

                if (s < H) {
                    Real *So = sb_cur + (s - 1) * 2 * PLANE;
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        tmem_st4(K2 + fcol(s - 1, 0) + r * VEC, out[r]);
                        if constexpr (C::KAHAN) tmem_st4(K2 + fcol(s - 1, 1) + r * VEC, cout[r]);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            prev[r][v] = out[r][v];
                            zmh[r][v] = zm[r][v];
                        }
                        if (r == 0 || r == RPT - 1) st_vec<Real>(So + own + r * W, out[r]);
                    }
                } else {
                    // I of the last step: the center of F_{H-1}'s window
                    Real vi[RPT][VEC];
                    Real vci[C::KAHAN ? RPT : 1][VEC];
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        tmem_ld4(K1 + fcol(H - 2, 0) + r * VEC, vi[r]);
                        if constexpr (C::KAHAN) tmem_ld4(K1 + fcol(H - 2, 1) + r * VEC, vci[r]);
                    }
                    tmem_wait_ld();
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        after_wait(vi[r]);
                        if constexpr (C::KAHAN) after_wait(vci[r]);
                    }
                    if (any_store && (FAST || (q >= kz0 && q < kz1))) {
                        const long long zoff = static_cast<long long>(q) * S.plane;
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            if (!store_row[r]) continue;
                            if (absorb) {
#pragma unroll
                                for (int v = 0; v < VEC; ++v) {
                                    vi[r][v] = mul_rn(vi[r][v], mq);
                                    if constexpr (C::KAHAN) vci[r][v] = mul_rn(vci[r][v], mq);
                                }
                            }
                            store_output_row<Real, C::KAHAN, VEC>(S, outR, outI, outCR, outCI,
                                                                  zoff + out0 + r * pitch, pitch,
                                                                  seam, xs, ys0 + r, out[r], vi[r],
                                                                  cout[r], vci[C::KAHAN ? r : 0]);
                        }
                    }
                }
            }
        };

        int ph = 0;   // it % 3: window slot of the old plane
        int dj = 0;   // TMEM slot of d at plane p (modulo NDT)
        // One plane of the z-march once its loads have landed: d to TMEM, the stages,
        // the ring heads.
        auto plane_body = [&](const int it) {
            const int p = L0 + it;
            tmem_wait_st();   // the previous iteration's window planes are in TMEM
            {
                // d at plane p moves to TMEM slot dj; its shared-memory slot is free
                // again once every thread has copied it
                Real dp[RPT][VEC];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    ld_vec<Real>(ringD + headD * PLANE + own + r * W, dp[r]);
                    tmem_st4(dcol(dj) + r * VEC, dp[r]);
                }
            }
            const Real *A0 = ringA + headA * SLOT;
            const Real *A1 = ringA + (headA >= 1 ? headA - 1 : headA - 1 + NR) * SLOT;
            const Real *A2 = ringA + (headA >= 2 ? headA - 2 : headA - 2 + NR) * SLOT;
            const Real *I1 = ringI + (headI >= 1 ? headI - 1 : headI - 1 + NI) * SLOT;
            const Real *sb_prev = sbuf + ((it - 1) & 1) * PLANE;
            Real *sb_cur = sbuf + (it & 1) * PLANE;
            // TMEM bases of the old, center and new window planes at this phase
            const uint32_t K0 = pbase(ph), K1 = pbase(ph == 2 ? 0 : ph + 1), K2 = pbase(ph == 0 ? 2 : ph - 1);
            const bool fast = !tile_walls && it >= 2 * H && p >= fast_lo && p < fast_hi &&
                              !(flux_owner && p >= kd + 2 && p <= kd + H);
            if (fast)
                stages(it, p, K0, K1, K2, dj, A0, A1, A2, I1, sb_prev, sb_cur, std::true_type{});
            else
                stages(it, p, K0, K1, K2, dj, A0, A1, A2, I1, sb_prev, sb_cur, std::false_type{});
            headA = headA + 1 == NR ? 0 : headA + 1;
            headI = headI + 1 == NI ? 0 : headI + 1;
            headD = headD + 1 == ND ? 0 : headD + 1;
            headB = headB + 1 == NB ? 0 : headB + 1;
            if (headB == 0) phase ^= 1u;
            ph = ph == 2 ? 0 : ph + 1;
            ++dj;   // slots are taken modulo NDT
        };

        if constexpr (!WS) {
            for (int it = 0; it < nit; ++it) {
                if (tid == 0) {
                    if (mbar_wait_bounded(&bars[headB], phase, wait_ns)) {
                        waited = it + 1;
                    } else {
                        atomicOr(status, 1);
                        s_abort = 1;
                    }
                }
                __syncthreads();   // plane L0 + it has landed; the previous iteration's reads are done
                if (s_abort) break;
                if (it + PF < nit) {
                    if (tid == 0) {
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        issue(it + PF, PF);
                    }
                    issued = it + PF + 1;
                }
                plane_body(it);
            }
        } else if (producer) {
            // Plane l goes to ring slots l mod NR / NI / ND and barrier slot
            // (gbase + l) mod NB.  Those slots last held plane l - NB (the R, I and d
            // rings are read up to 2, 1 and 0 planes after landing, so their depths
            // PF + 3, PF + 2, PF + 1 all free their slot after plane l - NB's
            // iteration): refill only once every compute warp has reported it done.
            if (lane == 0) {
                for (int l = 0; l < nit; ++l) {
                    const long long g = gbase + l;
                    if (l >= NB) {
                        const long long gd = g - NB;
                        const int w = mbar_wait_or_abort(&done[gd % NB], static_cast<uint32_t>((gd / NB) & 1),
                                                         wait_ns, abort_flag);
                        if (w <= 0) {
                            if (w == 0) atomicOr(status, 1);
                            s_abort = 1;
                            break;
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    issue_at(l);
                    issued = l + 1;
                }
            }
        } else {
            for (int it = 0; it < nit; ++it) {
                const long long g = gbase + it;
                // this plane's loads have landed, and both neighbouring warps are done
                // with the previous plane (their edge rows of the stage planes)
                int w = mbar_wait_or_abort(&bars[g % NB], static_cast<uint32_t>((g / NB) & 1), wait_ns,
                                           abort_flag);
                if (w > 0 && g > 0)
                    w = mbar_wait_or_abort(&nbr[2 * warp + ((g - 1) & 1)],
                                           static_cast<uint32_t>(((g - 1) >> 1) & 1), wait_ns, abort_flag);
                const bool expired = __any_sync(kFull, w == 0);
                if (!__all_sync(kFull, w > 0)) {   // one decision for the whole warp
                    if (lane == 0) {
                        if (expired) atomicOr(status, 1);
                        s_abort = 1;
                    }
                    break;
                }
                plane_body(it);
                __syncwarp();   // every lane's stage-plane rows are written
                if (lane == 0) {
                    mbar_arrive(&done[g % NB]);
                    if (warp > 0) mbar_arrive(&nbr[2 * (warp - 1) + (g & 1)]);
                    if (warp < NWC - 1) mbar_arrive(&nbr[2 * (warp + 1) + (g & 1)]);
                }
            }
        }

        __syncthreads();   // every thread has left the z-march: all read the same s_abort
        if (s_abort) {
            // wait (bounded) for the loads still in flight, then leave (freeing TMEM below).
            // With a producer warp, planes before issued - NB had their slots refilled,
            // which required every warp to have consumed them: only the last NB remain.
            if (WS ? (producer && lane == 0) : tid == 0) {
                for (int l = WS ? max(0, issued - NB) : waited; l < issued; ++l) {
                    const long long g = gbase + l;
                    if (!mbar_wait_bounded(&bars[g % NB], static_cast<uint32_t>((g / NB) & 1)))
                        atomicOr(status, 4);   // the CTA leaves with a load still in flight
                }
            }
            __syncthreads();
            break;
        }
        gbase += nit;
        tmem_wait_st();
        __syncthreads();
    }

    tmem_wait_st();
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(s_tmem, TS::NCOLS);
}

template <class C, bool WS>
cudaError_t launch_tmem_cfg(const StepLaunch &L)
{
    typedef TmemSync<C, WS> Y;
    static std::atomic<uint64_t> smem_allowed{0};   // one bit per device
    cudaError_t e = allow_dynamic_smem(fused_step_tmem_kernel<C, WS>, Y::SMEM, smem_allowed);
    if (e != cudaSuccess) return e;
    fused_step_tmem_kernel<C, WS><<<L.grid, Y::THREADS, Y::SMEM, L.stream>>>(
        L.members, L.work, L.counter, L.status, L.in_buf, L.wait_ns);
    return cudaGetLastError();
}

template <class C, bool WS>
void fill_tmem_config(StepConfig *cfg)
{
    cfg->tile_x = C::TX;
    cfg->tile_y = C::TY;
    cfg->box_x = C::W;
    cfg->box_y = C::ROWS;
    cfg->threads = TmemSync<C, WS>::THREADS;
    cfg->smem = TmemSync<C, WS>::SMEM;
    cfg->ctas_per_sm = C::MINB;
}

}  // namespace

#define TDSE_TMEM_VARIANT(FN, ...)                                                      \
    cudaError_t launch_##FN(const StepLaunch &L) { return launch_tmem_cfg<Cfg<__VA_ARGS__>, false>(L); } \
    void fill_##FN(StepConfig *cfg) { fill_tmem_config<Cfg<__VA_ARGS__>, false>(cfg); }
// the same kernel shape with a producer warp and neighbour barriers (TmemSync)
#define TDSE_TMEM_WS_VARIANT(FN, ...)                                                   \
    cudaError_t launch_##FN(const StepLaunch &L) { return launch_tmem_cfg<Cfg<__VA_ARGS__>, true>(L); } \
    void fill_##FN(StepConfig *cfg) { fill_tmem_config<Cfg<__VA_ARGS__>, true>(cfg); }

// Cfg<Real, 2T, threads per row, rows, rows per thread, Kahan, planes prefetched, CTAs per SM,
//     d kept in TMEM>
TDSE_TMEM_VARIANT(tmem_k32_t2_r32x1_pf2, float, 4, 16, 32, 1, true, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_k32_t2_r28x1_pf2, float, 4, 16, 28, 1, true, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_f32_t2_r32x2_pf2, float, 4, 16, 32, 2, false, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_f32_t2_r32x1_pf3, float, 4, 16, 32, 1, false, 3, 1, true)
TDSE_TMEM_VARIANT(tmem_f32_t2_r32x1_pf4, float, 4, 16, 32, 1, false, 4, 1, true)
TDSE_TMEM_VARIANT(tmem_k32_t2_r28x1_pf3, float, 4, 16, 28, 1, true, 3, 1, true)
// 32-wide boxes, two CTAs per SM: each CTA's per-plane barrier runs independently
TDSE_TMEM_VARIANT(tmem_k32_t2_w32_r28x1_pf2_b2, float, 4, 8, 28, 1, true, 2, 2, true)
TDSE_TMEM_VARIANT(tmem_k32_t2_w32_r32x1_pf2_b2, float, 4, 8, 32, 1, true, 2, 2, true)
TDSE_TMEM_VARIANT(tmem_f32_t2_w32_r32x1_pf4_b2, float, 4, 8, 32, 1, false, 4, 2, true)
TDSE_TMEM_VARIANT(tmem_f32_t2_w32_r32x1_pf3_b2, float, 4, 8, 32, 1, false, 3, 2, true)
// three and four steps per launch (H = 6, 8): the windows of 5 or 7 intermediate
// fields fill tensor memory, so one CTA per SM
TDSE_TMEM_VARIANT(tmem_k32_t3_w32_r32x1_pf2, float, 6, 8, 32, 1, true, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_k32_t4_w32_r32x1_pf2, float, 8, 8, 32, 1, true, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_f32_t3_r32x1_pf2, float, 6, 16, 32, 1, false, 2, 1, true)
TDSE_TMEM_VARIANT(tmem_f32_t4_w32_r40x1_pf2, float, 8, 8, 40, 1, false, 2, 1, true)
TDSE_TMEM_WS_VARIANT(ws_k32_t3_w32_r32x1_pf2, float, 6, 8, 32, 1, true, 2, 1, true)
TDSE_TMEM_WS_VARIANT(ws_f32_t3_r32x1_pf2, float, 6, 16, 32, 1, false, 2, 1, true)
// producer warp + neighbour barriers
TDSE_TMEM_WS_VARIANT(ws_k32_t2_w32_r32x1_pf2_b2, float, 4, 8, 32, 1, true, 2, 2, true)
TDSE_TMEM_WS_VARIANT(ws_k32_t2_r32x1_pf2, float, 4, 16, 32, 1, true, 2, 1, true)
TDSE_TMEM_WS_VARIANT(ws_f32_t2_w32_r32x1_pf3_b2, float, 4, 8, 32, 1, false, 3, 2, true)
TDSE_TMEM_WS_VARIANT(ws_f32_t2_w32_r32x1_pf4_b2, float, 4, 8, 32, 1, false, 4, 2, true)

}  // namespace tdse
