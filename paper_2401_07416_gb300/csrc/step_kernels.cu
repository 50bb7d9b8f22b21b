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
#include <type_traits>

#include "step_common.cuh"

namespace tdse {

// Variants of the tensor-memory window kernel (step_tmem.cu).
#define TDSE_TMEM_DECL(FN)                        \
    cudaError_t launch_##FN(const StepLaunch &L); \
    void fill_##FN(StepConfig *cfg);
TDSE_TMEM_DECL(tmem_k32_t2_r32x1_pf2)
TDSE_TMEM_DECL(tmem_k32_t2_r28x1_pf2)
TDSE_TMEM_DECL(tmem_f32_t2_r32x2_pf2)
TDSE_TMEM_DECL(tmem_f32_t2_r32x1_pf3)
TDSE_TMEM_DECL(tmem_f32_t2_r32x1_pf4)
TDSE_TMEM_DECL(tmem_k32_t2_r28x1_pf3)
TDSE_TMEM_DECL(tmem_k32_t2_w32_r28x1_pf2_b2)
TDSE_TMEM_DECL(tmem_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(tmem_f32_t2_w32_r32x1_pf4_b2)
TDSE_TMEM_DECL(tmem_f32_t2_w32_r32x1_pf3_b2)
TDSE_TMEM_DECL(tmem_k32_t3_w32_r32x1_pf2)
TDSE_TMEM_DECL(tmem_k32_t4_w32_r32x1_pf2)
TDSE_TMEM_DECL(tmem_f32_t3_r32x1_pf2)
TDSE_TMEM_DECL(tmem_f32_t4_w32_r40x1_pf2)
TDSE_TMEM_DECL(ws_k32_t3_w32_r32x1_pf2)
TDSE_TMEM_DECL(ws_f32_t3_r32x1_pf2)
TDSE_TMEM_DECL(slim_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(roll_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(split_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(split_f32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(roll_k32_t2_w32_r28x1_pf2_b2)
TDSE_TMEM_DECL(roll_f32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(roll_k32_t2_w32_r32x1_pf3_b2)
TDSE_TMEM_DECL(roll_k32_t2_r32x1_pf2)
TDSE_TMEM_DECL(roll_k32_t2_r32x1_pf3)
TDSE_TMEM_DECL(split_k32_t2_r32x1_pf2)
TDSE_TMEM_DECL(split_k32_t2_r32x1_pf3)
TDSE_TMEM_DECL(split_f32_t2_r32x1_pf2)
TDSE_TMEM_DECL(split_f32_t2_r32x1_pf3)
TDSE_TMEM_DECL(split_k32_t2_w72_r32x1_pf2)
TDSE_TMEM_DECL(split_f32_t2_w72_r32x1_pf2)
TDSE_TMEM_DECL(split_f32_t2_w72_r32x1_pf3)
TDSE_TMEM_DECL(roll_f32_t2_w32_r32x1_pf3_b2)
TDSE_TMEM_DECL(roll_f32_t2_r32x1_pf3)
TDSE_TMEM_DECL(hyb_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(hyb_f32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(ws_k32_t2_w32_r32x1_pf2_b2)
TDSE_TMEM_DECL(ws_k32_t2_r32x1_pf2)
TDSE_TMEM_DECL(ws_f32_t2_w32_r32x1_pf3_b2)
TDSE_TMEM_DECL(ws_f32_t2_w32_r32x1_pf4_b2)
#undef TDSE_TMEM_DECL

namespace {

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB)
    fused_step_kernel(const MemberDev *__restrict__ members, const WorkDev *__restrict__ work,
                      int *counter, int *status, int in_buf, unsigned long long wait_ns)
{
    static_assert(C::ROW_IN_WARP, "x neighbours by shuffles need each region row inside one warp");
    typedef typename C::Real Real;
    constexpr int H = C::H, VEC = C::VEC, W = C::W, ROWS = C::ROWS, PLANE = C::PLANE;
    constexpr int RPT = C::RPT, NB = C::NB, PF = C::PF, NR = C::NR, NI = C::NI, ND = C::ND;
    constexpr int NF = H > 1 ? H - 1 : 1;   // register windows for F_1 .. F_{H-1}
    constexpr int SLOT = C::NFC * PLANE;    // one ring slot: a field (and its compensation)
    constexpr int OFF_C = PLANE;            // compensation term within a slot
    // A f = cx sx + cy sy + cz sz + d f (s_a: neighbour sums).  FP64 (ALU-bound)
    // folds the accumulator into the FMA chain; FP32 keeps the increment separate
    // so that its rounding happens at the increment's scale.
    constexpr bool CHAIN = sizeof(Real) == 8 && !C::KAHAN;
    constexpr bool PAIRED = sizeof(Real) == 4;   // FP32 node updates in paired instructions

    extern __shared__ unsigned char smem_raw[];
    // pointer arithmetic on smem_raw keeps the shared address space visible to the compiler
    Real *ringA = reinterpret_cast<Real *>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    Real *ringI = ringA + NR * SLOT;
    Real *ringD = ringI + NI * SLOT;
    Real *sbuf = ringD + ND * PLANE;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sbuf + C::NSB * PLANE);
    __shared__ int s_item;
    __shared__ int s_abort;
    __shared__ ItemScalars S;

    const int tid = threadIdx.x;
    const int qx = tid % C::TPX;
    const int r0 = (tid / C::TPX) * RPT;                 // first region row of this thread
    const int warp_row0 = (tid >> 5) * C::RW;
    const int own = r0 * W + qx * VEC;                   // row r of this thread: own + r * W
    const int off_ym = (r0 > 0 ? r0 - 1 : r0) * W + qx * VEC;
    const int off_yp = (r0 + RPT < ROWS ? r0 + RPT : r0 + RPT - 1) * W + qx * VEC;

    if (tid == 0) {
        for (int b = 0; b < NB; ++b) mbar_init(&bars[b], 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();

    long long gbase = 0;   // loads issued by this CTA before the current item

    for (;;) {
        // thread 0 takes the next work item and stages the member's scalars in
        // shared memory (loop invariants then never come back from global memory)
        if (tid == 0) fetch_item(members, work, counter, in_buf, &s_item, S);
        __syncthreads();
        const int item = s_item;
        if (item >= work->total) break;
        const int m = S.m;
        const MemberDev &M = members[m];   // tensor maps only (thread 0)
        const int tile_x = S.tile_x, tile_y = S.tile_y, kz0 = S.kz0, kz1 = S.kz1;
        const int L0 = kz0 - H;                 // first plane loaded
        const int nit = (kz1 - kz0) + 2 * H;    // iterations (planes loaded)
        const int G = S.G, nx = S.nx, ny = S.ny, nz = S.nz;
        const int bx = G + tile_x * C::TX - C::HX;   // padded coordinates of the box
        const int by = G + tile_y * C::TY - H;
        const int xs = tile_x * C::TX - C::HX + qx * VEC;   // unpadded x of the first cell
        const int ys0 = tile_y * C::TY - H + r0;             // unpadded y of row 0
        const bool zper = S.per_z != 0;
        const int mlo = S.mask_lo, mhi = nz - S.mask_hi;    // planes outside [mlo, mhi) absorb
        const Real cx = static_cast<Real>(S.cx), cy = static_cast<Real>(S.cy),
                   cz = static_cast<Real>(S.cz);
        const float2 cx2 = make_float2(float(cx), float(cx)), cy2 = make_float2(float(cy), float(cy)),
                     cz2 = make_float2(float(cz), float(cz));
        const Real *maskz = reinterpret_cast<const Real *>(S.mask);
        const int kd = S.det_k;
        const bool flux_owner = kd >= kz0 && kd < kz1;

        // Cells outside the domain on a walled axis are kept at zero after every stage.
        auto inside = [&](int r, int v) {
            return (S.per_x || (xs + v >= 0 && xs + v < nx)) && (S.per_y || (ys0 + r >= 0 && ys0 + r < ny));
        };
        bool walls = false;
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
            for (int v = 0; v < VEC; ++v) walls |= !inside(r, v);
        const bool col_in = qx * VEC >= C::HX && qx * VEC < C::HX + C::TX && xs < nx;
        bool store_row[RPT];
        bool any_store = false;
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            store_row[r] = col_in && r0 + r >= H && r0 + r < H + C::TY && ys0 + r < ny;
            any_store |= store_row[r];
        }
        // output offsets within a plane (primary location; ghost copies of periodic axes
        // are added only on tiles that touch a seam)
        const long long pitch = S.pitch;
        const bool seam = (S.per_x && (xs < G || xs >= nx - G)) ||
                          (S.per_y && (ys0 < G || ys0 + RPT - 1 >= ny - G));
        Real *outR = reinterpret_cast<Real *>(S.outR);
        Real *outI = reinterpret_cast<Real *>(S.outI);
        Real *outCR = reinterpret_cast<Real *>(S.outCR);
        Real *outCI = reinterpret_cast<Real *>(S.outCI);
        const long long out0 = static_cast<long long>(ys0 + G) * pitch + (xs + G);

        // Register windows of F_1 .. F_{H-1}.  The z-march is unrolled by three and
        // the window slots are renamed rather than moved: in iteration `it`, once
        // stage f+1 has run, slot it % 3 of window f holds F_{f+1} at plane q-1
        // (old), slot (it+1) % 3 at q (center) and slot (it+2) % 3 at q+1 (new),
        // where q = p-f-2 is the plane stage f+2 works on.
        Real w[NF][3][RPT][VEC];
        Real cw[C::KAHAN ? NF : 1][3][RPT][VEC];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int k = 0; k < 3; ++k)
#pragma unroll
                for (int r = 0; r < RPT; ++r)
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        w[f][k][r][v] = Real(0);
                        if constexpr (C::KAHAN) cw[f][k][r][v] = Real(0);
                    }

        // Planes p whose stages all work on interior planes (no wall, absorbing
        // layer, detector or wrap) take a path without those checks; the
        // arithmetic is the same on both paths.
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

        if (tid == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int l = 0; l < PF && l < nit; ++l) issue(l, l);
        }
        int issued = min(PF, nit);
        int waited = 0;

        // The H stages of one iteration (plane p loaded, stage s on plane p - s).
        auto stages = [&](const int it, const int p, const Real *A0, const Real *A1,
                          const Real *A2, const Real *I1, const Real *sb_prev, Real *sb_cur,
                          auto PHc, auto FASTc) {
            constexpr int PH = decltype(PHc)::value;
            constexpr bool FAST = decltype(FASTc)::value;
            constexpr int K0 = PH, K1 = (PH + 1) % 3, K2 = (PH + 2) % 3;   // old, center, new
            const bool p_out = !FAST && !zper && (p < 0 || p >= nz);

            Real zmR[RPT][VEC];   // R at plane p-2: stage 1's z- neighbour, stage 2's accumulator
#pragma unroll
            for (int s = 1; s <= H; ++s) {
                if (!FAST && it < 2 * s) continue;                            // pipeline filling
                if (warp_row0 + C::RW <= s || warp_row0 >= ROWS - s) continue;  // rows outside the cone
                const int q = p - s;
                const bool odd = (s & 1) != 0;
                bool q_out = false, absorb = false;
                Real mq = Real(1);
                if constexpr (!FAST) {
                    q_out = !zper && (q < 0 || q >= nz);
                    int qm = q;                      // plane index inside [0, nz) (periodic z wraps)
                    if (zper) {
                        qm = q % nz;
                        if (qm < 0) qm += nz;
                    }
                    absorb = !q_out && (qm < mlo || qm >= mhi);
                    if (absorb) mq = maskz[qm];
                }
                int dslot = headD - s;
                if (dslot < 0) dslot += ND;
                const Real *Dp = ringD + dslot * PLANE;

                Real zm[RPT][VEC], c[RPT][VEC], zp[RPT][VEC], ym[VEC], yp[VEC], dd[RPT][VEC];
                if (s == 1) {
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        ld_vec<Real>(A2 + own + r * W, zmR[r]);
                        ld_vec<Real>(A1 + own + r * W, c[r]);
                        ld_vec<Real>(A0 + own + r * W, zp[r]);
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            zm[r][v] = zmR[r][v];
                            if (p_out) zp[r][v] = Real(0);
                        }
                    }
                    ld_vec<Real>(A1 + off_ym, ym);
                    ld_vec<Real>(A1 + off_yp, yp);
                } else {
                    const Real *Sp = sb_prev + (s - 2) * 2 * PLANE;
#pragma unroll
                    for (int r = 0; r < RPT; ++r)
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            zm[r][v] = w[s - 2][K0][r][v];
                            c[r][v] = w[s - 2][K1][r][v];
                            zp[r][v] = w[s - 2][K2][r][v];
                        }
                    ld_vec<Real>(Sp + off_ym, ym);
                    ld_vec<Real>(Sp + off_yp, yp);
                }
#pragma unroll
                for (int r = 0; r < RPT; ++r) ld_vec<Real>(Dp + own + r * W, dd[r]);

                // accumulator: the field two stages back at plane q
                Real acc[RPT][VEC], cacc[RPT][VEC];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    if (s == 1) {
                        ld_vec<Real>(I1 + own + r * W, acc[r]);
                        if constexpr (C::KAHAN) ld_vec<Real>(I1 + OFF_C + own + r * W, cacc[r]);
                    } else if (s == 2) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) acc[r][v] = zmR[r][v];
                        if constexpr (C::KAHAN) ld_vec<Real>(A2 + OFF_C + own + r * W, cacc[r]);
                    } else {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            acc[r][v] = w[s - 3][K0][r][v];
                            if constexpr (C::KAHAN) cacc[r][v] = cw[s - 3][K0][r][v];
                        }
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
                    if constexpr (PAIRED) {
                        update_row_f32<C::KAHAN, VEC>(
                            odd, c[r], xl, xr, r == 0 ? ym : c[r - 1], r == RPT - 1 ? yp : c[r + 1], zm[r],
                            zp[r], dd[r], acc[r], cacc[r], cx2, cy2, cz2, out[r], cout[r]);
                        continue;
                    }
#pragma unroll
                    for (int v = 0; v < VEC; ++v) {
                        const Real sx = (v == 0 ? xl : c[r][v - 1]) + (v == VEC - 1 ? xr : c[r][v + 1]);
                        const Real sy = (r == 0 ? ym[v] : c[r - 1][v]) + (r == RPT - 1 ? yp[v] : c[r + 1][v]);
                        const Real sz = zm[r][v] + zp[r][v];
                        if constexpr (CHAIN) {
                            const Real sg = odd ? Real(1) : Real(-1);
                            out[r][v] = fma(sg * cx, sx, fma(sg * cy, sy,
                                            fma(sg * cz, sz, fma(sg * dd[r][v], c[r][v], acc[r][v]))));
                        } else {
                            const Real delta = fma(cx, sx, fma(cy, sy, fma(cz, sz, dd[r][v] * c[r][v])));
                            const Real inc = odd ? delta : -delta;
                            if constexpr (C::KAHAN) {
                                const Real y = inc - cacc[r][v];
                                const Real t = acc[r][v] + y;
                                cout[r][v] = (t - acc[r][v]) - y;
                                out[r][v] = t;
                            } else {
                                out[r][v] = acc[r][v] + inc;
                            }
                        }
                    }
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
                        const Real zq = q_out ? Real(0) : Real(1);
#pragma unroll
                        for (int r = 0; r < RPT; ++r)
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                const Real keep = inside(r, v) ? Real(1) : Real(0);
                                out[r][v] *= keep * zq;
                                if constexpr (C::KAHAN) cout[r][v] *= keep * zq;
                            }
                    }

                    // detector flux of step (s+1)/2: R^n at planes kd, kd+1 and the new I
                    if (odd && flux_owner && q == kd + 1 && any_store) {
#pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            if (!store_row[r]) continue;
                            const int pix = (ys0 + r) * nx + xs;
#pragma unroll
                            for (int v = 0; v < VEC; ++v) {
                                // I at plane kd: the previous output of stage s
                                const Real ilo = s < H ? w[s - 1][K1][r][v] : Real(0);
                                const double j = S.cj * (static_cast<double>(zm[r][v]) * out[r][v] -
                                                         static_cast<double>(c[r][v]) * ilo);
                                S.flux[pix + v] += j * S.dt;
                                if (s == H - 1) S.jlast[pix + v] = j;
                            }
                        }
                    }
                }

                if (s < H) {
                    Real *So = sb_cur + (s - 1) * 2 * PLANE;
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            w[s - 1][K2][r][v] = out[r][v];
                            if constexpr (C::KAHAN) cw[s - 1][K2][r][v] = cout[r][v];
                        }
                        if (r == 0 || r == RPT - 1) st_vec<Real>(So + own + r * W, out[r]);
                    }
                } else if (any_store && (FAST || (q >= kz0 && q < kz1))) {
                    const long long zoff = static_cast<long long>(q) * S.plane;
#pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        if (!store_row[r]) continue;
                        Real vi[VEC], vci[VEC];
#pragma unroll
                        for (int v = 0; v < VEC; ++v) {
                            vi[v] = absorb ? mul_rn(w[H - 2][K1][r][v], mq) : w[H - 2][K1][r][v];
                            if constexpr (C::KAHAN)
                                vci[v] = absorb ? mul_rn(cw[H - 2][K1][r][v], mq) : cw[H - 2][K1][r][v];
                        }
                        store_output_row<Real, C::KAHAN, VEC>(S, outR, outI, outCR, outCI,
                                                              zoff + out0 + r * pitch, pitch, seam,
                                                              xs, ys0 + r, out[r], vi, cout[r], vci);
                    }
                }
            }
        };

        // One iteration: wait for plane L0 + it, refill the ring, run the stages.
        auto plane_step = [&](const int it, auto PHc) -> bool {
            const int p = L0 + it;
            if (tid == 0) {
                if (mbar_wait_bounded(&bars[headB], phase, wait_ns)) {
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
                    issue(it + PF, PF);
                }
                issued = it + PF + 1;
            }
            // R slots of planes p, p-1, p-2 and the I slot of plane p-1
            const Real *A0 = ringA + headA * SLOT;
            const Real *A1 = ringA + (headA >= 1 ? headA - 1 : headA - 1 + NR) * SLOT;
            const Real *A2 = ringA + (headA >= 2 ? headA - 2 : headA - 2 + NR) * SLOT;
            const Real *I1 = ringI + (headI >= 1 ? headI - 1 : headI - 1 + NI) * SLOT;
            const Real *sb_prev = sbuf + ((it - 1) & 1) * PLANE;   // + 2 (f) PLANE for F_{f+1}
            Real *sb_cur = sbuf + (it & 1) * PLANE;
            const bool fast = !tile_walls && it >= 2 * H && p >= fast_lo && p < fast_hi &&
                              !(flux_owner && p >= kd + 2 && p <= kd + H);
            if (fast)
                stages(it, p, A0, A1, A2, I1, sb_prev, sb_cur, PHc, std::true_type{});
            else
                stages(it, p, A0, A1, A2, I1, sb_prev, sb_cur, PHc, std::false_type{});
            headA = headA + 1 == NR ? 0 : headA + 1;
            headI = headI + 1 == NI ? 0 : headI + 1;
            headD = headD + 1 == ND ? 0 : headD + 1;
            headB = headB + 1 == NB ? 0 : headB + 1;
            if (headB == 0) phase ^= 1u;
            return true;
        };

        for (int it0 = 0; it0 < nit; it0 += 3) {
            if (!plane_step(it0, std::integral_constant<int, 0>{})) break;
            if (it0 + 1 >= nit || !plane_step(it0 + 1, std::integral_constant<int, 1>{})) break;
            if (it0 + 2 >= nit || !plane_step(it0 + 2, std::integral_constant<int, 2>{})) break;
        }

        if (s_abort) {
            // wait (bounded) for the loads still in flight, then leave
            if (tid == 0) {
                for (int l = waited; l < issued; ++l) {
                    const long long g = gbase + l;
                    if (!mbar_wait_bounded(&bars[g % NB], static_cast<uint32_t>((g / NB) & 1)))
                        atomicOr(status, 4);   // the CTA leaves with a load still in flight
                }
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
    static std::atomic<uint64_t> smem_allowed{0};   // one bit per device
    cudaError_t e = allow_dynamic_smem(fused_step_kernel<C>, C::SMEM, smem_allowed);
    if (e != cudaSuccess) return e;
    fused_step_kernel<C><<<L.grid, C::NT, C::SMEM, L.stream>>>(L.members, L.work, L.counter,
                                                               L.status, L.in_buf, L.wait_ns);
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
    cfg->ctas_per_sm = C::MINB;
}

struct Variant {
    int precision, tsteps;
    const char *name;
    void (*fill)(StepConfig *);
    cudaError_t (*launch)(const StepLaunch &);
};

#define TDSE_VARIANT(P, T, NAME, ...)                                                      \
    Variant{P, T, NAME, &fill_config<Cfg<__VA_ARGS__>>, &launch_cfg<Cfg<__VA_ARGS__>>}

// Kernel variants per (precision, fused steps): register-window kernels
// (TDSE_VARIANT: Cfg<Real, 2T, threads per row, rows, rows per thread, Kahan,
// planes prefetched, CTAs per SM>), tensor-memory-window kernels with run-time rings
// (step_tmem.cu: tmem_*, producer-warp ws_*) and with late loads and rolling slots
// (step_slim.cu: roll_*, split_*, slim_*, hyb_*).  The first entry of each
// (precision, steps) group is the default: the fastest on GB300 (512x512x1024 grid)
// at the makespan model's z-chunk.  The autotuner times every entry at several
// chunks; some (the one-CTA split forms) win only at chunks the model does not pick.
const Variant kVariants[] = {
    TDSE_VARIANT(1, 1, "f32_t1_w64_r24x2_pf2_b2", float, 2, 16, 24, 2, false, 2, 2),
    TDSE_VARIANT(1, 1, "f32_t1_w64_r48x2_pf2", float, 2, 16, 48, 2, false, 2),
    TDSE_VARIANT(1, 1, "f32_t1_w128_r24x2_pf2", float, 2, 32, 24, 2, false, 2),
    Variant{1, 2, "f32_t2_roll_w32_r32x1_pf2_b2", &fill_roll_f32_t2_w32_r32x1_pf2_b2, &launch_roll_f32_t2_w32_r32x1_pf2_b2},
    Variant{1, 2, "f32_t2_split_w32_r32x1_pf2_b2", &fill_split_f32_t2_w32_r32x1_pf2_b2, &launch_split_f32_t2_w32_r32x1_pf2_b2},
    Variant{1, 2, "f32_t2_split_r32x1_pf2", &fill_split_f32_t2_r32x1_pf2, &launch_split_f32_t2_r32x1_pf2},
    Variant{1, 2, "f32_t2_split_r32x1_pf3", &fill_split_f32_t2_r32x1_pf3, &launch_split_f32_t2_r32x1_pf3},
    Variant{1, 2, "f32_t2_roll_w32_r32x1_pf3_b2", &fill_roll_f32_t2_w32_r32x1_pf3_b2, &launch_roll_f32_t2_w32_r32x1_pf3_b2},
    Variant{1, 2, "f32_t2_tmem_w32_r32x1_pf3_b2", &fill_tmem_f32_t2_w32_r32x1_pf3_b2, &launch_tmem_f32_t2_w32_r32x1_pf3_b2},
    Variant{1, 2, "f32_t2_tmem_w32_r32x1_pf4_b2", &fill_tmem_f32_t2_w32_r32x1_pf4_b2, &launch_tmem_f32_t2_w32_r32x1_pf4_b2},
    Variant{1, 2, "f32_t2_roll_r32x1_pf3", &fill_roll_f32_t2_r32x1_pf3, &launch_roll_f32_t2_r32x1_pf3},
    Variant{1, 2, "f32_t2_tmem_r32x1_pf3", &fill_tmem_f32_t2_r32x1_pf3, &launch_tmem_f32_t2_r32x1_pf3},
    Variant{1, 2, "f32_t2_tmem_r32x1_pf4", &fill_tmem_f32_t2_r32x1_pf4, &launch_tmem_f32_t2_r32x1_pf4},
    Variant{1, 2, "f32_t2_tmem_r32x2_pf2", &fill_tmem_f32_t2_r32x2_pf2, &launch_tmem_f32_t2_r32x2_pf2},
    Variant{1, 2, "f32_t2_hyb_w32_r32x1_pf2_b2", &fill_hyb_f32_t2_w32_r32x1_pf2_b2, &launch_hyb_f32_t2_w32_r32x1_pf2_b2},
    Variant{1, 2, "f32_t2_ws_w32_r32x1_pf3_b2", &fill_ws_f32_t2_w32_r32x1_pf3_b2, &launch_ws_f32_t2_w32_r32x1_pf3_b2},
    Variant{1, 2, "f32_t2_ws_w32_r32x1_pf4_b2", &fill_ws_f32_t2_w32_r32x1_pf4_b2, &launch_ws_f32_t2_w32_r32x1_pf4_b2},
    TDSE_VARIANT(1, 2, "f32_t2_w64_r32x2_pf2", float, 4, 16, 32, 2, false, 2),
    Variant{1, 2, "f32_t2_split_w72_r32x1_pf2", &fill_split_f32_t2_w72_r32x1_pf2, &launch_split_f32_t2_w72_r32x1_pf2},
    Variant{1, 2, "f32_t2_split_w72_r32x1_pf3", &fill_split_f32_t2_w72_r32x1_pf3, &launch_split_f32_t2_w72_r32x1_pf3},
    TDSE_VARIANT(2, 1, "k32_t1_w64_r32x2_pf2", float, 2, 16, 32, 2, true, 2),
    TDSE_VARIANT(2, 1, "k32_t1_w64_r32x1_pf2", float, 2, 16, 32, 1, true, 2),
    Variant{2, 2, "k32_t2_roll_w32_r32x1_pf2_b2", &fill_roll_k32_t2_w32_r32x1_pf2_b2, &launch_roll_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_tmem_w32_r32x1_pf2_b2", &fill_tmem_k32_t2_w32_r32x1_pf2_b2, &launch_tmem_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_ws_r32x1_pf2", &fill_ws_k32_t2_r32x1_pf2, &launch_ws_k32_t2_r32x1_pf2},
    Variant{2, 2, "k32_t2_roll_r32x1_pf2", &fill_roll_k32_t2_r32x1_pf2, &launch_roll_k32_t2_r32x1_pf2},
    Variant{2, 2, "k32_t2_tmem_r28x1_pf2", &fill_tmem_k32_t2_r28x1_pf2, &launch_tmem_k32_t2_r28x1_pf2},
    Variant{2, 2, "k32_t2_tmem_w32_r28x1_pf2_b2", &fill_tmem_k32_t2_w32_r28x1_pf2_b2, &launch_tmem_k32_t2_w32_r28x1_pf2_b2},
    Variant{2, 2, "k32_t2_roll_w32_r28x1_pf2_b2", &fill_roll_k32_t2_w32_r28x1_pf2_b2, &launch_roll_k32_t2_w32_r28x1_pf2_b2},
    Variant{2, 2, "k32_t2_tmem_r32x1_pf2", &fill_tmem_k32_t2_r32x1_pf2, &launch_tmem_k32_t2_r32x1_pf2},
    Variant{2, 2, "k32_t2_tmem_r28x1_pf3", &fill_tmem_k32_t2_r28x1_pf3, &launch_tmem_k32_t2_r28x1_pf3},
    Variant{2, 2, "k32_t2_ws_w32_r32x1_pf2_b2", &fill_ws_k32_t2_w32_r32x1_pf2_b2, &launch_ws_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_slim_w32_r32x1_pf2_b2", &fill_slim_k32_t2_w32_r32x1_pf2_b2, &launch_slim_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_split_w32_r32x1_pf2_b2", &fill_split_k32_t2_w32_r32x1_pf2_b2, &launch_split_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_hyb_w32_r32x1_pf2_b2", &fill_hyb_k32_t2_w32_r32x1_pf2_b2, &launch_hyb_k32_t2_w32_r32x1_pf2_b2},
    Variant{2, 2, "k32_t2_roll_r32x1_pf3", &fill_roll_k32_t2_r32x1_pf3, &launch_roll_k32_t2_r32x1_pf3},
    Variant{2, 2, "k32_t2_split_r32x1_pf2", &fill_split_k32_t2_r32x1_pf2, &launch_split_k32_t2_r32x1_pf2},
    Variant{2, 2, "k32_t2_split_r32x1_pf3", &fill_split_k32_t2_r32x1_pf3, &launch_split_k32_t2_r32x1_pf3},
    Variant{2, 2, "k32_t2_roll_w32_r32x1_pf3_b2", &fill_roll_k32_t2_w32_r32x1_pf3_b2, &launch_roll_k32_t2_w32_r32x1_pf3_b2},
    TDSE_VARIANT(2, 2, "k32_t2_w64_r32x2_pf1", float, 4, 16, 32, 2, true, 1),
    Variant{2, 2, "k32_t2_split_w72_r32x1_pf2", &fill_split_k32_t2_w72_r32x1_pf2, &launch_split_k32_t2_w72_r32x1_pf2},
    Variant{1, 3, "f32_t3_tmem_r32x1_pf2", &fill_tmem_f32_t3_r32x1_pf2, &launch_tmem_f32_t3_r32x1_pf2},
    Variant{1, 3, "f32_t3_ws_r32x1_pf2", &fill_ws_f32_t3_r32x1_pf2, &launch_ws_f32_t3_r32x1_pf2},
    Variant{1, 4, "f32_t4_tmem_w32_r40x1_pf2", &fill_tmem_f32_t4_w32_r40x1_pf2, &launch_tmem_f32_t4_w32_r40x1_pf2},
    Variant{2, 3, "k32_t3_tmem_w32_r32x1_pf2", &fill_tmem_k32_t3_w32_r32x1_pf2, &launch_tmem_k32_t3_w32_r32x1_pf2},
    Variant{2, 3, "k32_t3_ws_w32_r32x1_pf2", &fill_ws_k32_t3_w32_r32x1_pf2, &launch_ws_k32_t3_w32_r32x1_pf2},
    Variant{2, 4, "k32_t4_tmem_w32_r32x1_pf2", &fill_tmem_k32_t4_w32_r32x1_pf2, &launch_tmem_k32_t4_w32_r32x1_pf2},
    TDSE_VARIANT(0, 1, "f64_t1_w64_r16x2_pf1_b2", double, 2, 32, 16, 2, false, 1, 2),
    TDSE_VARIANT(0, 1, "f64_t1_w64_r16x1_pf2", double, 2, 32, 16, 1, false, 2),
};

const Variant *find_variant(int precision, int tsteps, int variant)
{
    int k = 0;
    for (const Variant &v : kVariants)
        if (v.precision == precision && v.tsteps == tsteps && k++ == variant) return &v;
    return nullptr;
}

}  // namespace

int step_variant_count(int precision, int tsteps)
{
    int k = 0;
    for (const Variant &v : kVariants) k += (v.precision == precision && v.tsteps == tsteps);
    return k;
}

const char *step_variant_name(int precision, int tsteps, int variant)
{
    const Variant *v = find_variant(precision, tsteps, variant);
    return v ? v->name : nullptr;
}

bool step_config(int precision, int tsteps, int variant, StepConfig *cfg)
{
    const Variant *v = find_variant(precision, tsteps, variant);
    if (!v) return false;
    v->fill(cfg);
    return true;
}

cudaError_t launch_step(int precision, int tsteps, int variant, const StepLaunch &L)
{
    const Variant *v = find_variant(precision, tsteps, variant);
    return v ? v->launch(L) : cudaErrorInvalidValue;
}

}  // namespace tdse
