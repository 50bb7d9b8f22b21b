// C ABI of libtdse (declared in include/tdse.h): contexts, device memory,
// TMA descriptors, work planning and the launch sequence of tdse_step.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "tdse.h"
#include "tdse_internal.cuh"

using namespace tdse;

namespace {

constexpr int kRecCap = 256;        // observation records buffered on the device per member
constexpr int kRecLen = 6;
constexpr int kStatusLag = 2;       // observation points whose status copies may be outstanding
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;   // 2 s per wait for a tile's data

struct Member {
    tdse_params p;                  // resolved parameters
    MemberDev dev;                  // device pointers and geometry (tensor maps per config below)
    double *V64 = nullptr;          // FP64 potential, unpadded
    bool have_potential = false;
    bool have_state = false;
    std::vector<double> atoms;      // [n][4] if the potential came from atoms
    double soft_a2 = 0.25, r_cut = 0.0;
    double q0 = 0.0;                // Q at the last set_wavepacket / set_state
    std::vector<double> hist;       // 4 per record: step, Q, norm_paper, energy
    void *mask_inv = nullptr;       // reciprocal of the absorbing factor per plane (adjoint)
    double mask_min = 1.0;          // smallest factor, in the step's number format
    bool from_packet = false;       // the run started with tdse_set_wavepacket
    std::vector<std::pair<long long, double *>> ckpts;   // (step, FP64 R then I)
    double *frames = nullptr;       // detector density frames [frame_cap][ny][nx] (Eq. 15)
    int frame_cap = 0;
    std::vector<long long> frame_steps;   // step of each recorded frame
};

struct StepPlan {
    int tsteps = 0;
    int variant = 0;
    int chunk_request = 0;          // z-planes per work item requested (0: the makespan model's)
    int chunk = 0;                  // ... in use (the longest member's)
    StepConfig cfg{};
    MemberDev *d_members = nullptr; // members with tensor maps for this config's box
    WorkDev *d_work = nullptr;
    int grid = 0;
};

}  // namespace

struct tdse_ctx {
    std::vector<Member> m;
    int precision = 0, tblock = 1, obs_every = 20, ckpt_every = 0;
    bool tblock_auto = false;       // created with tblock = 0: tdse_autotune may change it
    tdse_alloc_fn alloc_fn = nullptr;
    tdse_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    cudaStream_t stream = nullptr;
    bool device_ready = false;
    std::vector<void *> allocations;
    StepPlan plans[kMaxTblock + 1];
    int *d_counter = nullptr;
    int *d_status = nullptr;
    // Status word copies taken at observation points (pinned host slots, one event
    // each), read by the host without stalling the stream.
    int *h_status = nullptr;
    cudaEvent_t status_ev[kStatusLag] = {};
    long long status_step[kStatusLag] = {};
    int status_head = 0, status_pending = 0;
    bool failed = false;                           // a step kernel timed out or the run diverged
    unsigned long long wait_ns = kDefaultWaitNs;   // limit of each wait for a tile's data
    double *d_partials = nullptr;
    // batched reductions (more than one member): each member's block slice
    std::vector<ObsSlice> obs_slices;
    ObsSlice *d_obs_slices = nullptr;
    int obs_blocks = 0;
    double *d_records = nullptr;    // [B][kRecCap][kRecLen]
    int cur = 0;                    // ping-pong buffer holding the state
    long long step = 0;
    int sms = 0;
    bool profiling = false;
    tdse_profile prof{};
    std::vector<cudaEvent_t> event_pool;           // reused timing events
    struct Interval {
        int start, stop;                           // indices into event_pool
        int kind;                                  // 0: step launches, 1: reductions, 2: backward steps
        int launches, depth;                       // step launches timed together, their depth
    };
    std::vector<Interval> pending;
    size_t events_used = 0;
    bool graphs = true;                            // replay step segments as CUDA graphs
    bool adjoint_fused = false;                    // one z-march per backward step (else three passes)
    cudaStream_t gstream = nullptr;                // capture/replay stream
    cudaEvent_t gev[2] = {nullptr, nullptr};
    struct GraphEntry {
        int nsteps, parity, tblock;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graph_cache;
    double tuned_ms_per_step[kMaxTblock + 1] = {};
    std::string err;
};

namespace {

const char *kVersion = "libtdse 1.0 (sm_103a)";

tdse_status fail(tdse_ctx *c, tdse_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

#define CUDA_TRY(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, TDSE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                 \
    } while (0)

#define TRY(expr)                                                                            \
    do {                                                                                     \
        tdse_status s_ = (expr);                                                             \
        if (s_ != TDSE_OK) return s_;                                                        \
    } while (0)

size_t elem_size(int precision) { return precision == TDSE_FP64 ? 8 : 4; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

tdse_status dalloc(tdse_ctx *c, size_t bytes, void **out)
{
    void *p = nullptr;
    if (c->alloc_fn) {
        p = c->alloc_fn(bytes, c->alloc_user);
        if (!p) return fail(c, TDSE_ENOMEM, "allocator returned NULL for %zu bytes", bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess)
            return fail(c, TDSE_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    c->allocations.push_back(p);
    CUDA_TRY(c, cudaMemsetAsync(p, 0, bytes, c->stream));
    *out = p;
    return TDSE_OK;
}

void dfree(tdse_ctx *c, void *p)
{
    if (!p) return;
    auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
    if (it != c->allocations.end()) c->allocations.erase(it);
    if (c->free_fn)
        c->free_fn(p, c->alloc_user);
    else
        cudaFree(p);
}

tdse_status validate(tdse_ctx *c, const tdse_params &q, int idx)
{
    if (q.nx < 4 || q.ny < 1 || q.nz < 3)
        return fail(c, TDSE_EINVAL, "member %d: grid %dx%dx%d too small (nx >= 4, nz >= 3)", idx,
                    q.nx, q.ny, q.nz);
    if (q.nx % 4 != 0) return fail(c, TDSE_EINVAL, "member %d: nx=%d is not a multiple of 4", idx, q.nx);
    // per-plane indices (pixels, ghost cells, plane offsets inside a kernel) are 32-bit
    if (static_cast<long long>(q.nx + 2 * kGhost + 32) * (q.ny + 2 * kGhost) > (1LL << 30))
        return fail(c, TDSE_EINVAL, "member %d: an xy plane of %dx%d nodes exceeds 2^30 (padded)", idx,
                    q.nx, q.ny);
    if (!(q.hx > 0 && q.hy > 0 && q.hz > 0))
        return fail(c, TDSE_EINVAL, "member %d: spacings must be positive", idx);
    for (int a = 0; a < 3; ++a)
        if (q.bc[a] != TDSE_BC_PERIODIC && q.bc[a] != TDSE_BC_DIRICHLET)
            return fail(c, TDSE_EINVAL, "member %d: bad boundary flag on axis %d", idx, a);
    if ((q.bc[0] == TDSE_BC_PERIODIC && q.nx < kGhost) || (q.bc[1] == TDSE_BC_PERIODIC && q.ny < kGhost))
        return fail(c, TDSE_EINVAL, "member %d: periodic axis shorter than %d nodes", idx, kGhost);
    if (q.mask_lo < 0 || q.mask_hi < 0 || q.mask_lo + q.mask_hi > q.nz)
        return fail(c, TDSE_EINVAL, "member %d: absorbing layers exceed nz", idx);
    if (q.det_k < -1 || q.det_k > q.nz - 2)
        return fail(c, TDSE_EINVAL, "member %d: det_k=%d outside [-1, nz-2]", idx, q.det_k);
    // free-particle stability of the leapfrog: dt * max eigenvalue of H / hbar < 2
    const double emax = 2.0 * q.hbar / q.mass *
                        (1.0 / (q.hx * q.hx) + 1.0 / (q.hy * q.hy) + 1.0 / (q.hz * q.hz));
    if (!(q.dt > 0) || q.dt * emax >= 2.0)
        return fail(c, TDSE_EINVAL, "member %d: dt=%g violates dt*max|E|/hbar < 2 (max %g)", idx,
                    q.dt, 2.0 / emax);
    if (q.mask_kind != TDSE_MASK_COS2 && q.mask_kind != TDSE_MASK_CAP)
        return fail(c, TDSE_EINVAL, "member %d: unknown mask_kind %d", idx, q.mask_kind);
    if (q.mask_kind == TDSE_MASK_CAP && !(q.mask_eta >= 0.0))
        return fail(c, TDSE_EINVAL, "member %d: negative absorbing strength", idx);
    for (int r : q.reserved)
        if (r != 0) return fail(c, TDSE_EINVAL, "member %d: reserved fields must be zero", idx);
    return TDSE_OK;
}

tdse_status check_member(tdse_ctx *c, int member)
{
    if (!c) return TDSE_EINVAL;
    if (member < 0 || member >= static_cast<int>(c->m.size()))
        return fail(c, TDSE_EINVAL, "member %d out of range [0, %zu)", member, c->m.size());
    return TDSE_OK;
}

tdse_status encode_map(tdse_ctx *c, CUtensorMap *map, const Member &mb, void *ptr, int box_x,
                       int box_y)
{
    auto fn = encode_fn();
    if (!fn) return fail(c, TDSE_ECUDA, "cuTensorMapEncodeTiled unavailable");
    const size_t es = elem_size(c->precision);
    const MemberDev &d = mb.dev;
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(d.nx + 2 * d.G),
                          static_cast<cuuint64_t>(d.ny + 2 * d.G), static_cast<cuuint64_t>(d.nz)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(d.pitch) * es,
                             static_cast<cuuint64_t>(d.plane) * es};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(box_x), static_cast<cuuint32_t>(box_y), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, es == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                    3, ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(c, TDSE_ECUDA, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return TDSE_OK;
}

// z-chunk length minimising the estimated makespan ceil(items / P) * (L + 4T) of
// the dynamically scheduled work list (an item of L planes takes L + 2H = L + 4T
// iterations: its pipeline fills over the 2T half-step stages at each end).
int choose_chunk(const std::vector<int> &tiles, const std::vector<int> &nz, int tsteps, int P)
{
    int nzmax = *std::max_element(nz.begin(), nz.end());
    double best = 1e300;
    int bestL = nzmax;
    for (int L = 8; L <= nzmax; ++L) {
        long long items = 0;
        for (size_t i = 0; i < tiles.size(); ++i) items += static_cast<long long>(tiles[i]) * ((nz[i] + L - 1) / L);
        const double span = static_cast<double>((items + P - 1) / P) * (L + 4.0 * tsteps);
        if (span < best - 1e-9 || (std::fabs(span - best) < 1e-9 && L > bestL)) {
            best = span;
            bestL = L;
        }
    }
    return bestL;
}

void drop_graphs(tdse_ctx *c)
{
    for (auto &g : c->graph_cache) cudaGraphExecDestroy(g.exec);
    c->graph_cache.clear();
}

// Build (or rebuild) the launch plan of the fused step with T steps per launch
// and the given kernel variant: tensor maps with the variant's box, the work list.
tdse_status build_plan(tdse_ctx *c, int T, int variant)
{
    const int B = static_cast<int>(c->m.size());
    StepPlan &pl = c->plans[T];
    StepConfig cfg;
    if (!step_config(c->precision, T, variant, &cfg))
        return fail(c, TDSE_EINVAL, "no kernel variant %d for precision %d with %d fused steps",
                    variant, c->precision, T);
    std::vector<MemberDev> hm(B);
    WorkDev w{};
    w.nmembers = B;
    std::vector<int> tiles(B), nzs(B);
    for (int i = 0; i < B; ++i) {
        const Member &mb = c->m[i];
        hm[i] = mb.dev;
        MemberDev &d = hm[i];
        for (int b = 0; b < 2; ++b) {
            TRY(encode_map(c, &d.tm_R[b], mb, d.R[b], cfg.box_x, cfg.box_y));
            TRY(encode_map(c, &d.tm_I[b], mb, d.I[b], cfg.box_x, cfg.box_y));
            if (c->precision == TDSE_FP32_KAHAN) {
                TRY(encode_map(c, &d.tm_cR[b], mb, d.cR[b], cfg.box_x, cfg.box_y));
                TRY(encode_map(c, &d.tm_cI[b], mb, d.cI[b], cfg.box_x, cfg.box_y));
            }
        }
        TRY(encode_map(c, &d.tm_d, mb, d.d, cfg.box_x, cfg.box_y));
        w.tiles_x[i] = (d.nx + cfg.tile_x - 1) / cfg.tile_x;
        w.tiles_y[i] = (d.ny + cfg.tile_y - 1) / cfg.tile_y;
        tiles[i] = w.tiles_x[i] * w.tiles_y[i];
        nzs[i] = d.nz;
    }
    int dev = 0;
    CUDA_TRY(c, cudaGetDevice(&dev));
    CUDA_TRY(c, cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev));
    const int P = c->sms * std::max(1, cfg.ctas_per_sm);
    const int L = pl.chunk_request > 0 ? pl.chunk_request : choose_chunk(tiles, nzs, T, P);
    int total = 0;
    for (int i = 0; i < B; ++i) {
        w.item_begin[i] = total;
        w.chunk[i] = std::min(L, nzs[i]);
        total += tiles[i] * ((nzs[i] + w.chunk[i] - 1) / w.chunk[i]);
    }
    w.item_begin[B] = total;
    w.total = total;
    if (!pl.d_members) {
        void *p = nullptr;
        TRY(dalloc(c, sizeof(MemberDev) * B, &p));
        pl.d_members = static_cast<MemberDev *>(p);
        TRY(dalloc(c, sizeof(WorkDev), &p));
        pl.d_work = static_cast<WorkDev *>(p);
    }
    CUDA_TRY(c, cudaMemcpyAsync(pl.d_members, hm.data(), sizeof(MemberDev) * B,
                                cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(pl.d_work, &w, sizeof(WorkDev), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    pl.tsteps = T;
    pl.variant = variant;
    pl.chunk = L;
    pl.cfg = cfg;
    pl.grid = std::min(total, P);
    drop_graphs(c);
    return TDSE_OK;
}

// Plans of every fused depth that has kernel variants for the context's precision.
tdse_status build_plans(tdse_ctx *c)
{
    for (int T = 1; T <= kMaxTblock; ++T)
        if (step_variant_count(c->precision, T) > 0) TRY(build_plan(c, T, 0));
    return TDSE_OK;
}

// Allocate every device buffer of the context (first call only).
tdse_status ensure_device(tdse_ctx *c)
{
    if (c->device_ready) return TDSE_OK;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return fail(c, TDSE_ECUDA, "no CUDA device available");
    const size_t es = elem_size(c->precision);
    for (Member &mb : c->m) {
        MemberDev &d = mb.dev;
        const size_t fbytes = static_cast<size_t>(d.plane) * d.nz * es;
        void *p;
        for (int b = 0; b < 2; ++b) {
            TRY(dalloc(c, fbytes, &p)); d.R[b] = p;
            TRY(dalloc(c, fbytes, &p)); d.I[b] = p;
            if (c->precision == TDSE_FP32_KAHAN) {
                TRY(dalloc(c, fbytes, &p)); d.cR[b] = p;
                TRY(dalloc(c, fbytes, &p)); d.cI[b] = p;
            }
        }
        TRY(dalloc(c, fbytes, &p)); d.d = p;
        const size_t cells = static_cast<size_t>(d.nx) * d.ny * d.nz;
        TRY(dalloc(c, cells * sizeof(double), &p)); mb.V64 = static_cast<double *>(p);
        TRY(dalloc(c, static_cast<size_t>(d.nx) * d.ny * sizeof(double), &p)); d.flux = static_cast<double *>(p);
        TRY(dalloc(c, static_cast<size_t>(d.nx) * d.ny * sizeof(double), &p)); d.jlast = static_cast<double *>(p);
        // absorbing factor per plane at depth dep = 1..W into a layer of W planes:
        // cos^2(eta (pi/2) dep / W), or exp(-W(dep) dt / hbar) with the quadratic
        // W(dep) = eta (dep / W)^2 of Eq. 10 (operator split)
        std::vector<double> M(d.nz, 1.0);
        const tdse_params &q = mb.p;
        auto factor = [&](int dep, int W) {
            if (q.mask_kind == TDSE_MASK_CAP) {
                const double u = static_cast<double>(dep) / W;
                return std::exp(-q.mask_eta * u * u * q.dt / q.hbar);
            }
            const double s = std::cos(q.mask_eta * 0.5 * M_PI * dep / W);
            return s * s;
        };
        for (int k = 0; k < d.nz; ++k) {
            if (q.mask_lo > 0 && k < q.mask_lo) M[k] = factor(q.mask_lo - k, q.mask_lo);
            if (q.mask_hi > 0 && k >= d.nz - q.mask_hi)
                M[k] = factor(k - (d.nz - q.mask_hi) + 1, q.mask_hi);
        }
        TRY(dalloc(c, d.nz * es, &p)); d.mask = p;
        TRY(dalloc(c, d.nz * es, &p)); mb.mask_inv = p;
        // the factor in the step's number format, and its reciprocal (rounded once
        // from the exact reciprocal of that factor)
        std::vector<float> Mf(M.begin(), M.end()), Mfi(d.nz);
        std::vector<double> Mi(d.nz);
        for (int k = 0; k < d.nz; ++k) {
            Mi[k] = 1.0 / M[k];
            Mfi[k] = static_cast<float>(1.0 / static_cast<double>(Mf[k]));
            mb.mask_min = std::min(mb.mask_min, es == 8 ? M[k] : static_cast<double>(Mf[k]));
        }
        CUDA_TRY(c, cudaMemcpyAsync(d.mask, es == 8 ? static_cast<const void *>(M.data()) : Mf.data(),
                                    d.nz * es, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(mb.mask_inv, es == 8 ? static_cast<const void *>(Mi.data()) : Mfi.data(),
                                    d.nz * es, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    void *p;
    TRY(dalloc(c, sizeof(int), &p)); c->d_counter = static_cast<int *>(p);
    TRY(dalloc(c, sizeof(int), &p)); c->d_status = static_cast<int *>(p);
    CUDA_TRY(c, cudaHostAlloc(reinterpret_cast<void **>(&c->h_status), kStatusLag * sizeof(int),
                              cudaHostAllocDefault));
    for (int k = 0; k < kStatusLag; ++k)
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->status_ev[k], cudaEventDisableTiming));
    // each member's reduction blocks, one slice after the other (batched launches)
    c->obs_slices.resize(c->m.size());
    c->obs_blocks = 0;
    for (size_t i = 0; i < c->m.size(); ++i) {
        ObsSlice &sl = c->obs_slices[i];
        observables_shape(c->m[i].dev, c->precision, &sl.nparts, &sl.zch);
        sl.block_begin = c->obs_blocks;
        sl.q_ref = 0.0;
        c->obs_blocks += sl.nparts;
    }
    TRY(dalloc(c, static_cast<size_t>(std::max(kObsParts, c->obs_blocks)) * kObsPartialsPerBlock * sizeof(double),
               &p));
    c->d_partials = static_cast<double *>(p);
    TRY(dalloc(c, c->obs_slices.size() * sizeof(ObsSlice), &p));
    c->d_obs_slices = static_cast<ObsSlice *>(p);
    TRY(dalloc(c, c->m.size() * kRecCap * kRecLen * sizeof(double), &p));
    c->d_records = static_cast<double *>(p);
    TRY(build_plans(c));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->device_ready = true;
    return TDSE_OK;
}

tdse_status fill_all_ghosts(tdse_ctx *c, Member &mb, int buf)
{
    const int es = static_cast<int>(elem_size(c->precision));
    CUDA_TRY(c, launch_fill_ghosts(mb.dev, mb.dev.R[buf], es, c->stream));
    CUDA_TRY(c, launch_fill_ghosts(mb.dev, mb.dev.I[buf], es, c->stream));
    if (c->precision == TDSE_FP32_KAHAN) {
        CUDA_TRY(c, launch_fill_ghosts(mb.dev, mb.dev.cR[buf], es, c->stream));
        CUDA_TRY(c, launch_fill_ghosts(mb.dev, mb.dev.cI[buf], es, c->stream));
    }
    return TDSE_OK;
}

// Observation of member i at the current step into record slot `slot`.
tdse_status observe(tdse_ctx *c, int i, int slot, double q_ref)
{
    Member &mb = c->m[i];
    double *rec = c->d_records + (static_cast<size_t>(i) * kRecCap + slot) * kRecLen;
    CUDA_TRY(c, launch_observables(mb.dev, c->precision, c->cur, c->d_partials, rec, c->d_status,
                                   q_ref, c->step, c->stream));
    return TDSE_OK;
}

tdse_status drain_records(tdse_ctx *c, int nrec)
{
    if (nrec <= 0) return TDSE_OK;
    std::vector<double> host(c->m.size() * kRecCap * kRecLen);
    CUDA_TRY(c, cudaMemcpyAsync(host.data(), c->d_records, host.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i < c->m.size(); ++i)
        for (int r = 0; r < nrec; ++r) {
            const double *x = &host[(i * kRecCap + r) * kRecLen];
            c->m[i].hist.insert(c->m[i].hist.end(), {x[0], x[1], x[2], x[3]});
        }
    return TDSE_OK;
}

// Status word -> status code.  A set word leaves the context failed: the state
// is not a result of the scheme any more.
tdse_status status_error(tdse_ctx *c, int st, long long step)
{
    if (st == 0) return TDSE_OK;
    c->failed = true;
    if (st & 5)
        return fail(c, TDSE_ETIMEOUT, "a bounded wait for a tile's data in the step kernel expired "
                    "(seen by step %lld)%s", step,
                    (st & 4) ? "; a load was still in flight when its CTA left" : "");
    return fail(c, TDSE_EUNSTABLE, "non-finite values or growth of Q detected (seen at the "
                "observation of step %lld)", step);
}

tdse_status check_status(tdse_ctx *c)
{
    int st = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->status_pending = 0;   // every outstanding copy is older than this read
    return status_error(c, st, c->step);
}

// Look at the status copies of earlier observation points whose events have
// completed (oldest first); with `wait_oldest`, wait for the oldest one.
tdse_status poll_status(tdse_ctx *c, bool wait_oldest)
{
    while (c->status_pending > 0) {
        const int k = (c->status_head - c->status_pending + kStatusLag) % kStatusLag;
        const cudaError_t q = wait_oldest ? cudaEventSynchronize(c->status_ev[k])
                                          : cudaEventQuery(c->status_ev[k]);
        if (q == cudaErrorNotReady) return TDSE_OK;
        if (q != cudaSuccess) return fail(c, TDSE_ECUDA, "status event: %s", cudaGetErrorString(q));
        wait_oldest = false;
        --c->status_pending;
        TRY(status_error(c, c->h_status[k], c->status_step[k]));
    }
    return TDSE_OK;
}

// Copy the status word at this observation point into the next pinned slot; at
// most kStatusLag copies stay outstanding, so the host learns of a failure at
// most kStatusLag observation intervals after the point that recorded it.
tdse_status post_status(tdse_ctx *c)
{
    if (c->status_pending == kStatusLag) TRY(poll_status(c, true));
    const int k = c->status_head;
    CUDA_TRY(c, cudaMemcpyAsync(&c->h_status[k], c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                                c->stream));
    CUDA_TRY(c, cudaEventRecord(c->status_ev[k], c->stream));
    c->status_step[k] = c->step;
    c->status_head = (k + 1) % kStatusLag;
    ++c->status_pending;
    return TDSE_OK;
}

tdse_status check_usable(tdse_ctx *c)
{
    if (c->failed)
        return fail(c, TDSE_ESTATE, "the context failed earlier (a step kernel timed out or the run "
                    "diverged); its state is not a result of the scheme: destroy it");
    return TDSE_OK;
}

tdse_status next_event(tdse_ctx *c, int *idx)
{
    if (c->events_used == c->event_pool.size()) {
        cudaEvent_t e;
        CUDA_TRY(c, cudaEventCreate(&e));
        c->event_pool.push_back(e);
    }
    *idx = static_cast<int>(c->events_used++);
    return TDSE_OK;
}

// Open a timed interval on the stream (profiling only); returns the start index.
tdse_status timer_start(tdse_ctx *c, int *start)
{
    *start = -1;
    if (!c->profiling) return TDSE_OK;
    TRY(next_event(c, start));
    CUDA_TRY(c, cudaEventRecord(c->event_pool[*start], c->stream));
    return TDSE_OK;
}

// Close the interval: `launches` step launches of `depth` fused steps (kind 0),
// or one round of reductions (kind 1).
tdse_status timer_stop(tdse_ctx *c, int start, int kind, int launches = 1, int depth = 0)
{
    if (start < 0) return TDSE_OK;
    int stop;
    TRY(next_event(c, &stop));
    CUDA_TRY(c, cudaEventRecord(c->event_pool[stop], c->stream));
    c->pending.push_back({start, stop, kind, launches, depth});
    return TDSE_OK;
}

// Accumulate the recorded intervals (call after the stream has been synchronised).
tdse_status resolve_timers(tdse_ctx *c)
{
    for (const tdse_ctx::Interval &iv : c->pending) {
        float ms = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&ms, c->event_pool[iv.start], c->event_pool[iv.stop]));
        if (iv.kind == 0) {
            c->prof.step_launches += iv.launches;
            c->prof.step_ms += ms;
            if (iv.depth >= 1 && iv.depth <= TDSE_MAX_TBLOCK) {
                c->prof.launches_at_depth[iv.depth] += iv.launches;
                c->prof.ms_at_depth[iv.depth] += ms;
            }
        } else if (iv.kind == 1) {
            c->prof.reduce_launches += 2;   // the reduction and its finalize (all members at once)
            c->prof.reduce_ms += ms;
        } else {
            c->prof.adjoint_steps += iv.launches;
            c->prof.adjoint_ms += ms;
        }
    }
    c->pending.clear();
    c->events_used = 0;
    return TDSE_OK;
}

// Profile bookkeeping of one step launch of depth T (nodes per launch, last depth).
void note_launch(tdse_ctx *c, int T)
{
    if (!c->profiling) return;
    long long cells = 0;
    for (const Member &mb : c->m) cells += static_cast<long long>(mb.dev.nx) * mb.dev.ny * mb.dev.nz;
    c->prof.cells_per_launch = cells;
    c->prof.steps_per_launch = T;
}

// One fused launch of T steps; with profiling on and `timed`, bracketed by events.
tdse_status launch_fused(tdse_ctx *c, int T, bool timed = true)
{
    StepPlan &pl = c->plans[T];
    StepLaunch L;
    L.members = pl.d_members;
    L.work = pl.d_work;
    L.counter = c->d_counter;
    L.status = c->d_status;
    L.in_buf = c->cur;
    L.wait_ns = c->wait_ns;
    L.grid = pl.grid;
    L.block = pl.cfg.threads;
    L.smem = pl.cfg.smem;
    L.stream = c->stream;
    CUDA_TRY(c, cudaMemsetAsync(c->d_counter, 0, sizeof(int), c->stream));
    int t0 = -1;
    if (timed) TRY(timer_start(c, &t0));
    CUDA_TRY(c, launch_step(c->precision, T, pl.variant, L));
    TRY(timer_stop(c, t0, 0, 1, T));
    note_launch(c, T);
    c->cur ^= 1;
    c->step += T;
    return TDSE_OK;
}

// Depth of the launches of an n-step segment: T = tblock while at least T steps
// remain, then single steps.
int segment_depth(const tdse_ctx *c, long long left) { return left >= c->tblock ? c->tblock : 1; }

// Issue the fused launches of `nsteps` steps (no observation in between); with
// profiling on, each launch is timed by its own events.
tdse_status issue_segment(tdse_ctx *c, long long nsteps, bool timed = true)
{
    while (nsteps > 0) {
        const int T = segment_depth(c, nsteps);
        TRY(launch_fused(c, T, timed));
        nsteps -= T;
    }
    return TDSE_OK;
}

// Same launches, replayed from a captured CUDA graph keyed by (steps, ping-pong
// parity, fused depth).  Captured on a private stream that is ordered after and
// before the context's stream with events.
tdse_status ensure_gstream(tdse_ctx *c)
{
    if (!c->gstream) {
        CUDA_TRY(c, cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->gev[0], cudaEventDisableTiming));
        CUDA_TRY(c, cudaEventCreateWithFlags(&c->gev[1], cudaEventDisableTiming));
    }
    return TDSE_OK;
}

// Launch an instantiated graph on the private stream, ordered after and before
// the context's stream.
tdse_status replay_graph(tdse_ctx *c, cudaGraphExec_t exec)
{
    CUDA_TRY(c, cudaEventRecord(c->gev[0], c->stream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->gstream, c->gev[0], 0));
    CUDA_TRY(c, cudaGraphLaunch(exec, c->gstream));
    CUDA_TRY(c, cudaEventRecord(c->gev[1], c->gstream));
    CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->gev[1], 0));
    return TDSE_OK;
}

tdse_status run_segment(tdse_ctx *c, long long nsteps)
{
    // profiled segments are replayed (and timed as a whole) only when all their
    // launches have one depth, so that the time can be attributed to it
    const bool uniform = nsteps % c->tblock == 0;
    if (!c->graphs || nsteps <= 0 || (c->profiling && !uniform)) return issue_segment(c, nsteps);
    TRY(ensure_gstream(c));
    cudaGraphExec_t exec = nullptr;
    for (auto &g : c->graph_cache)
        if (g.nsteps == nsteps && g.parity == c->cur && g.tblock == c->tblock) exec = g.exec;
    const int cur0 = c->cur;
    const long long step0 = c->step;
    if (!exec) {
        cudaStream_t user = c->stream;
        c->stream = c->gstream;
        cudaGraph_t graph = nullptr;
        CUDA_TRY(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
        tdse_status st = issue_segment(c, nsteps, false);
        cudaError_t e = cudaStreamEndCapture(c->gstream, &graph);
        c->stream = user;
        c->cur = cur0;
        c->step = step0;
        if (st != TDSE_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (st != TDSE_OK) return st;
            return fail(c, TDSE_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(c, TDSE_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
        c->graph_cache.push_back({static_cast<int>(nsteps), cur0, c->tblock, exec});
    }
    int t0 = -1;
    TRY(timer_start(c, &t0));
    TRY(replay_graph(c, exec));
    TRY(timer_stop(c, t0, 0, static_cast<int>(nsteps / c->tblock), c->tblock));
    // the replay advanced the state exactly like issue_segment would have
    long long left = nsteps;
    while (left > 0) {
        const int T = segment_depth(c, left);
        note_launch(c, T);
        c->cur ^= 1;
        c->step += T;
        left -= T;
    }
    return TDSE_OK;
}

tdse_status observe_all(tdse_ctx *c, int slot)
{
    int t0;
    TRY(timer_start(c, &t0));
    if (c->m.size() == 1) {
        TRY(observe(c, 0, slot, c->m[0].q0));
    } else {   // every member in one reduction launch and one finalize launch
        CUDA_TRY(c, launch_observables_batch(c->plans[1].d_members, c->d_obs_slices,
                                             static_cast<int>(c->m.size()), c->obs_blocks, c->precision,
                                             c->cur, c->d_partials, c->d_records + slot * kRecLen,
                                             static_cast<long long>(kRecCap) * kRecLen, c->d_status, c->step,
                                             c->stream));
    }
    TRY(timer_stop(c, t0, 1));
    return TDSE_OK;
}

void clear_checkpoints(tdse_ctx *c, Member &mb)
{
    for (auto &ck : mb.ckpts) dfree(c, ck.second);
    mb.ckpts.clear();
}

// FP64 copy of member i's state at the current step (value - compensation in Kahan mode).
tdse_status save_checkpoint(tdse_ctx *c, Member &mb)
{
    const size_t cells = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz;
    void *p = nullptr;
    TRY(dalloc(c, 2 * cells * sizeof(double), &p));
    double *buf = static_cast<double *>(p);
    CUDA_TRY(c, launch_get_state(mb.dev, buf, buf + cells, c->precision, c->cur, c->stream));
    mb.ckpts.push_back({c->step, buf});
    return TDSE_OK;
}

// Observation of member i right now (synchronous) into rec[kRecLen].
tdse_status current_obs(tdse_ctx *c, int i, double *rec)
{
    TRY(observe(c, i, kRecCap - 1, 0.0));
    CUDA_TRY(c, cudaMemcpyAsync(rec, c->d_records + (static_cast<size_t>(i) * kRecCap + kRecCap - 1) * kRecLen,
                                kRecLen * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TDSE_OK;
}

// Record the detector density frame of member i at the current step, if the
// member has a frame buffer with room left.
tdse_status capture_frame(tdse_ctx *c, int i)
{
    Member &mb = c->m[i];
    if (!mb.frames || static_cast<int>(mb.frame_steps.size()) >= mb.frame_cap) return TDSE_OK;
    const size_t npix = static_cast<size_t>(mb.dev.nx) * mb.dev.ny;
    CUDA_TRY(c, launch_frame(mb.dev, c->precision, c->cur, mb.frames + mb.frame_steps.size() * npix,
                             c->stream));
    mb.frame_steps.push_back(c->step);
    return TDSE_OK;
}

tdse_status reset_run(tdse_ctx *c, int i)
{
    Member &mb = c->m[i];
    const size_t pix = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * sizeof(double);
    CUDA_TRY(c, cudaMemsetAsync(mb.dev.flux, 0, pix, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(mb.dev.jlast, 0, pix, c->stream));
    mb.hist.clear();
    mb.have_state = true;
    clear_checkpoints(c, mb);
    if (c->ckpt_every > 0) TRY(save_checkpoint(c, mb));
    double rec[kRecLen];
    TRY(current_obs(c, i, rec));
    mb.q0 = rec[1];
    c->obs_slices[i].q_ref = mb.q0;
    CUDA_TRY(c, cudaMemcpy(c->d_obs_slices + i, &c->obs_slices[i], sizeof(ObsSlice), cudaMemcpyHostToDevice));
    mb.hist.insert(mb.hist.end(), {static_cast<double>(c->step), rec[1], rec[2], rec[3]});
    mb.frame_steps.clear();
    TRY(capture_frame(c, i));
    return TDSE_OK;
}

tdse_status potential_to_d(tdse_ctx *c, Member &mb, const double *V_dev)
{
    const int es = static_cast<int>(elem_size(c->precision));
    CUDA_TRY(c, launch_build_d(mb.dev, es, V_dev, mb.V64, c->stream));
    CUDA_TRY(c, launch_fill_ghosts(mb.dev, mb.dev.d, es, c->stream));
    mb.have_potential = true;
    return TDSE_OK;
}

}  // namespace

namespace {

const char kMagic[8] = {'T', 'D', 'S', 'E', 'S', 'T', '0', '1'};

bool same_grid(const tdse_params &a, const tdse_params &b)
{
    return a.nx == b.nx && a.ny == b.ny && a.nz == b.nz && a.hx == b.hx && a.hy == b.hy &&
           a.hz == b.hz && a.dt == b.dt && a.hbar == b.hbar && a.mass == b.mass &&
           a.bc[0] == b.bc[0] && a.bc[1] == b.bc[1] && a.bc[2] == b.bc[2] &&
           a.mask_lo == b.mask_lo && a.mask_hi == b.mask_hi && a.mask_eta == b.mask_eta &&
           a.mask_kind == b.mask_kind && a.det_k == b.det_k && a.precision == b.precision;
}

template <typename T>
bool put(FILE *f, const T *p, size_t n) { return fwrite(p, sizeof(T), n, f) == n; }
template <typename T>
bool get(FILE *f, T *p, size_t n) { return fread(p, sizeof(T), n, f) == n; }

}  // namespace

extern "C" {

const char *tdse_version(void) { return kVersion; }

const char *tdse_last_error(const tdse_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : "NULL context";
}

tdse_status tdse_create(const tdse_params *p, int batch, tdse_ctx **out)
{
    if (!p || !out || batch < 1 || batch > 256) return TDSE_EINVAL;
    *out = nullptr;
    tdse_ctx *c = new tdse_ctx;
    c->precision = p[0].precision;
    if (c->precision < TDSE_FP64 || c->precision > TDSE_FP32_KAHAN) {
        delete c;
        return TDSE_EINVAL;
    }
    int tb = p[0].tblock;
    if (tb <= 0) tb = (c->precision == TDSE_FP64) ? 1 : 2;
    if (tb > kMaxTblock || step_variant_count(c->precision, tb) == 0) {
        delete c;
        return TDSE_EINVAL;
    }
    c->tblock = tb;
    c->tblock_auto = p[0].tblock <= 0;
    c->obs_every = p[0].obs_every > 0 ? p[0].obs_every : 20;
    c->ckpt_every = std::max(0, p[0].ckpt_every);
    for (int i = 0; i < batch; ++i) {
        Member mb;
        mb.p = p[i];
        tdse_params &q = mb.p;
        if (q.precision != p[0].precision || q.tblock != p[0].tblock ||
            q.obs_every != p[0].obs_every || q.ckpt_every != p[0].ckpt_every) {
            delete c;
            return TDSE_EINVAL;
        }
        if (q.hbar <= 0) q.hbar = 1.0;
        if (q.mass <= 0) q.mass = 1.0;
        if (q.dt <= 0) {
            const double h = std::min(q.hx, std::min(q.hy, q.hz));
            q.dt = q.mass / (5.0 * q.hbar) * h * h;   // Eq. 11
        }
        tdse_status st = validate(c, q, i);
        if (st != TDSE_OK) {
            delete c;
            return st;
        }
        MemberDev &d = mb.dev;
        memset(&d, 0, sizeof d);
        d.nx = q.nx;
        d.ny = q.ny;
        d.nz = q.nz;
        d.G = kGhost;
        d.pitch = ((q.nx + 2 * kGhost) + 31) / 32 * 32;
        d.prow = q.ny + 2 * kGhost;
        d.plane = static_cast<long long>(d.pitch) * d.prow;
        d.per_x = q.bc[0] == TDSE_BC_PERIODIC;
        d.per_y = q.bc[1] == TDSE_BC_PERIODIC;
        d.per_z = q.bc[2] == TDSE_BC_PERIODIC;
        d.det_k = q.det_k;
        d.mask_lo = q.mask_lo;
        d.mask_hi = q.mask_hi;
        d.cx = q.hbar * q.dt / (2.0 * q.mass * q.hx * q.hx);
        d.cy = q.hbar * q.dt / (2.0 * q.mass * q.hy * q.hy);
        d.cz = q.hbar * q.dt / (2.0 * q.mass * q.hz * q.hz);
        d.cv = q.dt / q.hbar;
        d.cj = q.hbar / (q.mass * q.hz);
        d.dt = q.dt;
        d.hx = q.hx;
        d.hy = q.hy;
        d.hz = q.hz;
        d.hbar = q.hbar;
        c->m.push_back(mb);
    }
    *out = c;
    return TDSE_OK;
}

tdse_status tdse_set_allocator(tdse_ctx *c, tdse_alloc_fn alloc, tdse_free_fn free_fn, void *user)
{
    if (!c) return TDSE_EINVAL;
    if (c->device_ready) return fail(c, TDSE_ESTATE, "allocator must be set before the first allocation");
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(c, TDSE_EINVAL, "alloc and free callbacks must both be set or both NULL");
    c->alloc_fn = alloc;
    c->free_fn = free_fn;
    c->alloc_user = user;
    return TDSE_OK;
}

tdse_status tdse_set_stream(tdse_ctx *c, void *stream)
{
    if (!c) return TDSE_EINVAL;
    c->stream = static_cast<cudaStream_t>(stream);
    return TDSE_OK;
}

tdse_status tdse_set_potential(tdse_ctx *c, int member, const double *V, int on_device)
{
    TRY(check_member(c, member));
    if (!V) return fail(c, TDSE_EINVAL, "V is NULL");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    const size_t bytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz * sizeof(double);
    const double *Vd = V;
    if (!on_device) {
        // Pinned (page-locked, mapped) host V: the d kernel reads it over the host link
        // itself and writes the resident FP64 copy on the way.  A copy-engine transfer
        // issued right after a long run of kernels was measured at 135-155 ms for 2.1 GB
        // where the kernel's reads took 19-25 ms (10 ms either way otherwise).  Pageable
        // host V goes through a copy into the resident copy first.
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, V) == cudaSuccess && a.type == cudaMemoryTypeHost &&
            a.devicePointer != nullptr) {
            Vd = static_cast<const double *>(a.devicePointer);
        } else {
            cudaGetLastError();   // a failed query leaves no error behind
            CUDA_TRY(c, cudaMemcpyAsync(mb.V64, V, bytes, cudaMemcpyHostToDevice, c->stream));
            Vd = mb.V64;
        }
    }
    tdse_status st = potential_to_d(c, mb, Vd);
    if (!on_device) CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // the host buffer is free again
    mb.atoms.clear();
    return st;
}

tdse_status tdse_set_potential_grid(tdse_ctx *c, int member, const double *Vc, int cnx, int cny,
                                    int cnz, const double cell[3], const double origin[3],
                                    int on_device)
{
    TRY(check_member(c, member));
    if (!Vc || !cell || !origin) return fail(c, TDSE_EINVAL, "NULL argument");
    if (cnx < 1 || cny < 1 || cnz < 1) return fail(c, TDSE_EINVAL, "empty cell lattice");
    for (int a = 0; a < 3; ++a)
        if (!(cell[a] > 0 && std::isfinite(cell[a]) && std::isfinite(origin[a])))
            return fail(c, TDSE_EINVAL, "cell lengths must be positive and finite, origin finite");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    const size_t cbytes = static_cast<size_t>(cnx) * cny * cnz * sizeof(double);
    void *tmpc = nullptr, *tab = nullptr;
    auto release = [&]() {
        cudaStreamSynchronize(c->stream);
        dfree(c, tmpc);
        dfree(c, tab);
    };
    const double *Vcd = Vc;
    tdse_status st = TDSE_OK;
    if (!on_device) {
        if ((st = dalloc(c, cbytes, &tmpc)) != TDSE_OK) return st;
        if (cudaMemcpyAsync(tmpc, Vc, cbytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            release();
            return fail(c, TDSE_ECUDA, "copy of the cell potential failed");
        }
        Vcd = static_cast<const double *>(tmpc);
    }
    if ((st = dalloc(c, interp_scratch_bytes(mb.dev), &tab)) != TDSE_OK) {
        release();
        return st;
    }
    // the interpolated V is written straight into the resident FP64 copy
    if (launch_interp(mb.dev, mb.p.hx, mb.p.hy, mb.p.hz, Vcd, cnx, cny, cnz, cell, origin, tab,
                      mb.V64, c->stream) != cudaSuccess) {
        release();
        return fail(c, TDSE_ECUDA, "interpolation kernel failed");
    }
    st = potential_to_d(c, mb, mb.V64);
    release();
    mb.atoms.clear();
    return st;
}

tdse_status tdse_set_atoms(tdse_ctx *c, int member, int n, const double *xyzZ, double soft_a2,
                           double r_cut)
{
    TRY(check_member(c, member));
    if (n < 0 || (n > 0 && !xyzZ)) return fail(c, TDSE_EINVAL, "bad atom list");
    if (!(soft_a2 > 0)) return fail(c, TDSE_EINVAL, "soft_a2 must be positive");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    const MemberDev &d = mb.dev;
    if (r_cut <= 0) {
        double rc = 0;
        bool any = false;
        const double L[3] = {d.nx * d.hx, d.ny * d.hy, d.nz * d.hz};
        const int per[3] = {d.per_x, d.per_y, d.per_z};
        for (int a = 0; a < 3; ++a)
            if (per[a]) {
                rc = any ? std::min(rc, 0.5 * L[a]) : 0.5 * L[a];
                any = true;
            }
        r_cut = rc;
    }
    void *A = nullptr, *AC = nullptr;
    TRY(dalloc(c, std::max<size_t>(1, 4 * static_cast<size_t>(n)) * sizeof(double), &A));
    TRY(dalloc(c, atom_cell_bytes(n), &AC));
    if (n > 0)
        CUDA_TRY(c, cudaMemcpyAsync(A, xyzZ, 4 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    // every node's V is written straight into the resident FP64 copy
    CUDA_TRY(c, launch_potential_atoms(d, static_cast<double *>(A), n, soft_a2, r_cut, mb.V64, AC,
                                       c->precision, c->stream));
    tdse_status st = potential_to_d(c, mb, mb.V64);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, A);
    dfree(c, AC);
    TRY(st);
    mb.atoms.assign(xyzZ, xyzZ + 4 * n);
    mb.soft_a2 = soft_a2;
    mb.r_cut = r_cut;
    return TDSE_OK;
}

tdse_status tdse_set_wavepacket(tdse_ctx *c, int member, const double r0[3], const double sigma[3],
                                const double k0[3])
{
    TRY(check_member(c, member));
    if (!r0 || !sigma || !k0) return fail(c, TDSE_EINVAL, "NULL packet parameter");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    if (!mb.have_potential) TRY(potential_to_d(c, mb, nullptr));   // V = 0
    void *scratch = nullptr;
    TRY(dalloc(c, packet_scratch_bytes(mb.dev), &scratch));
    CUDA_TRY(c, launch_packet_start(mb.dev, mb.V64, r0, sigma, k0, scratch, c->precision, c->cur,
                                    c->stream));
    TRY(fill_all_ghosts(c, mb, c->cur));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, scratch);
    mb.from_packet = true;
    return reset_run(c, member);
}

tdse_status tdse_set_state(tdse_ctx *c, int member, const double *R, const double *I, int on_device)
{
    TRY(check_member(c, member));
    if (!R || !I) return fail(c, TDSE_EINVAL, "NULL state");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    if (!mb.have_potential) TRY(potential_to_d(c, mb, nullptr));
    const size_t bytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz * sizeof(double);
    const double *Rd = R, *Id = I;
    void *tR = nullptr, *tI = nullptr;
    if (!on_device) {
        TRY(dalloc(c, bytes, &tR));
        TRY(dalloc(c, bytes, &tI));
        CUDA_TRY(c, cudaMemcpyAsync(tR, R, bytes, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(tI, I, bytes, cudaMemcpyHostToDevice, c->stream));
        Rd = static_cast<double *>(tR);
        Id = static_cast<double *>(tI);
    }
    CUDA_TRY(c, launch_set_state(mb.dev, Rd, Id, c->precision, c->cur, c->stream));
    TRY(fill_all_ghosts(c, mb, c->cur));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, tR);
    dfree(c, tI);
    mb.from_packet = false;
    return reset_run(c, member);
}

tdse_status tdse_step(tdse_ctx *c, long long nsteps)
{
    if (!c || nsteps < 0) return TDSE_EINVAL;
    TRY(check_usable(c));
    for (size_t i = 0; i < c->m.size(); ++i)
        if (!c->m[i].have_state)
            return fail(c, TDSE_ESTATE, "member %zu has no state (call tdse_set_wavepacket)", i);
    TRY(ensure_device(c));
    int nrec = 0;
    long long left = nsteps;
    tdse_status st = TDSE_OK;
    while (left > 0 && st == TDSE_OK) {
        long long seg = std::min(left, c->obs_every - (c->step % c->obs_every));
        if (c->ckpt_every > 0) seg = std::min(seg, c->ckpt_every - (c->step % c->ckpt_every));
        TRY(run_segment(c, seg));
        left -= seg;
        if (c->step % c->obs_every == 0) {
            TRY(observe_all(c, nrec));
            for (size_t i = 0; i < c->m.size(); ++i) TRY(capture_frame(c, static_cast<int>(i)));
            ++nrec;
            // posting may wait for (and report) an earlier point's status
            if ((st = post_status(c)) != TDSE_OK) break;
            if (nrec == kRecCap) {
                TRY(drain_records(c, nrec));
                nrec = 0;
            }
        }
        if (c->ckpt_every > 0 && c->step % c->ckpt_every == 0)
            for (Member &mb : c->m) TRY(save_checkpoint(c, mb));
        // a failure seen at an earlier observation point ends the call there
        // (at most kStatusLag observation intervals later), not after nsteps
        st = poll_status(c, false);
    }
    if (st != TDSE_OK) {
        cudaStreamSynchronize(c->stream);
        const std::string why = c->err;
        drain_records(c, nrec);
        resolve_timers(c);
        c->status_pending = 0;
        c->err = why;
        return st;
    }
    TRY(drain_records(c, nrec));
    TRY(check_status(c));
    return resolve_timers(c);
}

tdse_status tdse_observables(tdse_ctx *c, int member, tdse_obs *out)
{
    TRY(check_member(c, member));
    if (!out) return fail(c, TDSE_EINVAL, "NULL output");
    Member &mb = c->m[member];
    if (!mb.have_state) return fail(c, TDSE_ESTATE, "member has no state");
    double rec[kRecLen];
    TRY(current_obs(c, member, rec));
    out->Q = rec[1];
    out->norm_paper = rec[2];
    out->energy = rec[3];
    out->flux = rec[4];
    out->flux_integrated = rec[5];
    out->step = c->step;
    out->t = c->step * mb.p.dt;
    return TDSE_OK;
}

tdse_status tdse_set_frame_capacity(tdse_ctx *c, int member, int capacity)
{
    TRY(check_member(c, member));
    Member &mb = c->m[member];
    if (mb.p.det_k < 0) return fail(c, TDSE_EINVAL, "member %d has no detector plane", member);
    if (capacity < 0) return fail(c, TDSE_EINVAL, "negative frame capacity");
    TRY(ensure_device(c));
    dfree(c, mb.frames);
    mb.frames = nullptr;
    mb.frame_cap = 0;
    mb.frame_steps.clear();
    if (capacity > 0) {
        void *p = nullptr;
        TRY(dalloc(c, static_cast<size_t>(capacity) * mb.dev.nx * mb.dev.ny * sizeof(double), &p));
        mb.frames = static_cast<double *>(p);
        mb.frame_cap = capacity;
    }
    return TDSE_OK;
}

tdse_status tdse_get_frames(tdse_ctx *c, int member, double *frames, long long *steps, int cap,
                            int *count, int on_device)
{
    TRY(check_member(c, member));
    const Member &mb = c->m[member];
    const int n = static_cast<int>(mb.frame_steps.size());
    if (count) *count = n;
    const int k = std::min(std::max(cap, 0), n);
    if (steps && k > 0) memcpy(steps, mb.frame_steps.data(), k * sizeof(long long));
    if (frames && k > 0) {
        const size_t bytes = static_cast<size_t>(k) * mb.dev.nx * mb.dev.ny * sizeof(double);
        CUDA_TRY(c, cudaMemcpyAsync(frames, mb.frames, bytes,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    }
    return TDSE_OK;
}

tdse_status tdse_get_obs_history(tdse_ctx *c, int member, double *out, int cap, int *count)
{
    TRY(check_member(c, member));
    const std::vector<double> &h = c->m[member].hist;
    const int n = static_cast<int>(h.size() / 4);
    if (count) *count = n;
    if (out && cap > 0) memcpy(out, h.data(), std::min(cap, n) * 4 * sizeof(double));
    return TDSE_OK;
}

tdse_status tdse_get_state(tdse_ctx *c, int member, double *R, double *I, int on_device)
{
    TRY(check_member(c, member));
    Member &mb = c->m[member];
    if (!mb.have_state) return fail(c, TDSE_ESTATE, "member has no state");
    const size_t bytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz * sizeof(double);
    if (on_device) {
        CUDA_TRY(c, launch_get_state(mb.dev, R, I, c->precision, c->cur, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return TDSE_OK;
    }
    void *tR = nullptr, *tI = nullptr;
    if (R) TRY(dalloc(c, bytes, &tR));
    if (I) TRY(dalloc(c, bytes, &tI));
    CUDA_TRY(c, launch_get_state(mb.dev, static_cast<double *>(tR), static_cast<double *>(tI),
                                 c->precision, c->cur, c->stream));
    if (R) CUDA_TRY(c, cudaMemcpyAsync(R, tR, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (I) CUDA_TRY(c, cudaMemcpyAsync(I, tI, bytes, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    dfree(c, tR);
    dfree(c, tI);
    return TDSE_OK;
}

tdse_status tdse_get_flux_map(tdse_ctx *c, int member, double *F, int on_device)
{
    TRY(check_member(c, member));
    if (!F) return fail(c, TDSE_EINVAL, "NULL output");
    TRY(ensure_device(c));
    Member &mb = c->m[member];
    const size_t bytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * sizeof(double);
    CUDA_TRY(c, cudaMemcpyAsync(F, mb.dev.flux, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TDSE_OK;
}

tdse_status tdse_get_potential(tdse_ctx *c, int member, double *V, int on_device)
{
    TRY(check_member(c, member));
    if (!V) return fail(c, TDSE_EINVAL, "NULL output");
    Member &mb = c->m[member];
    if (!mb.have_potential) return fail(c, TDSE_ESTATE, "member has no potential");
    const size_t bytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz * sizeof(double);
    CUDA_TRY(c, cudaMemcpyAsync(V, mb.V64, bytes,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return TDSE_OK;
}

tdse_status tdse_adjoint(tdse_ctx *c, int member, const double *dL_dF, double *dL_dV,
                         double *dL_datoms, int on_device)
{
    TRY(check_member(c, member));
    TRY(check_usable(c));
    if (!dL_dF) return fail(c, TDSE_EINVAL, "dL_dF is NULL");
    Member &mb = c->m[member];
    if (!mb.have_state) return fail(c, TDSE_ESTATE, "member has no state");
    if (c->ckpt_every <= 0 || mb.ckpts.empty())
        return fail(c, TDSE_ESTATE, "no checkpoints: create the context with ckpt_every > 0");
    if (dL_datoms && mb.atoms.empty())
        return fail(c, TDSE_ESTATE, "dL_datoms requested but the potential did not come from atoms");
    if (!(mb.mask_min > 0.0))
        return fail(c, TDSE_EINVAL, "an absorbing factor is 0 (in the step's number format): "
                                    "the backward steps cannot undo it");
    const MemberDev &d = mb.dev;
    const size_t cells = static_cast<size_t>(d.nx) * d.ny * d.nz;
    const size_t npix = static_cast<size_t>(d.nx) * d.ny;
    const int elem = c->precision == TDSE_FP64 ? 8 : 4;
    std::vector<void *> tmp;
    auto alloc = [&](size_t bytes, void **p) -> tdse_status {
        tdse_status st = dalloc(c, bytes, p);
        if (st == TDSE_OK) tmp.push_back(*p);
        return st;
    };
    auto cleanup = [&]() {
        cudaStreamSynchronize(c->stream);
        for (void *p : tmp) dfree(c, p);
    };
    void *R, *I, *P, *Q, *gV, *w, *gF, *cur, *Ist;
    void *R2 = nullptr, *I2 = nullptr, *P2 = nullptr, *Q2 = nullptr;
    tdse_status st = TDSE_OK;
    if ((st = alloc(cells * elem, &R)) || (st = alloc(cells * elem, &I)) ||
        (st = alloc(cells * elem, &P)) || (st = alloc(cells * elem, &Q)) ||
        (st = alloc(cells * 8, &gV)) || (st = alloc(npix * 8, &w)) || (st = alloc(npix * 8, &gF)) ||
        (st = alloc(2 * cells * 8, &cur)) || (st = alloc(2 * npix * elem, &Ist)) ||
        (c->adjoint_fused && ((st = alloc(cells * elem, &R2)) || (st = alloc(cells * elem, &I2)) ||
                              (st = alloc(cells * elem, &P2)) || (st = alloc(cells * elem, &Q2))))) {
        cleanup();
        return st;
    }
    const AdjointBuffers base{R, I, P, Q, R2, I2, P2, Q2, static_cast<double *>(gV),
                              static_cast<double *>(w), mb.mask_inv, Ist, mb.V64};
    // The fused step reads one buffer set and writes the other: `par` says which set
    // holds the current state (the three-pass step works in place, par stays 0).
    int par = 0;
    auto view = [&]() {
        AdjointBuffers v = base;
        if (par) {
            std::swap(v.R, v.R2);
            std::swap(v.I, v.I2);
            std::swap(v.P, v.P2);
            std::swap(v.Q, v.Q2);
        }
        return v;
    };
    auto issue_step = [&](cudaStream_t s) -> cudaError_t {
        const cudaError_t e = adjoint_backward_step(d, elem, view(), s);
        if (base.R2) par ^= 1;
        return e;
    };
    // backward steps of one checkpoint segment, replayed from a CUDA graph per segment
    // length and starting buffer set (the buffers are this call's, so the graphs are too)
    struct AdjGraph {
        long long nsteps;
        int par;
        cudaGraphExec_t exec;
    };
    std::vector<AdjGraph> graphs;
    auto back_steps_untimed = [&](long long nsteps) -> tdse_status {
        if (nsteps <= 0) return TDSE_OK;
        if (!c->graphs) {
            for (long long k = 0; k < nsteps; ++k) CUDA_TRY(c, issue_step(c->stream));
            return TDSE_OK;
        }
        TRY(ensure_gstream(c));
        cudaGraphExec_t exec = nullptr;
        for (auto &g : graphs)
            if (g.nsteps == nsteps && g.par == par) exec = g.exec;
        const int par0 = par;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            CUDA_TRY(c, cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (long long k = 0; k < nsteps && e == cudaSuccess; ++k) e = issue_step(c->gstream);
            par = par0;
            const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &graph);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e != cudaSuccess)
                return fail(c, TDSE_ECUDA, "adjoint graph capture failed: %s", cudaGetErrorString(e));
            graphs.push_back({nsteps, par0, exec});
        }
        TRY(replay_graph(c, exec));
        if (base.R2 && (nsteps & 1)) par ^= 1;
        return TDSE_OK;
    };
    auto back_steps = [&](long long nsteps) -> tdse_status {
        int t0 = -1;
        TRY(timer_start(c, &t0));
        TRY(back_steps_untimed(nsteps));
        return timer_stop(c, t0, 2, static_cast<int>(nsteps), 0);
    };
    auto drop_graphs = [&]() {
        for (auto &g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
    };
    auto run = [&]() -> tdse_status {
        CUDA_TRY(c, cudaMemcpyAsync(gF, dL_dF, npix * 8,
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                    c->stream));
        CUDA_TRY(c, adjoint_flux_weights(d, static_cast<double *>(gF), base.w, c->stream));
        // start from the latest state, then walk the checkpoints backwards
        double *cur64 = static_cast<double *>(cur);
        CUDA_TRY(c, launch_get_state(d, cur64, cur64 + cells, c->precision, c->cur, c->stream));
        CUDA_TRY(c, adjoint_load_state(d, elem, view(), cur64, cur64 + cells, c->stream));
        long long n = c->step;
        for (int k = static_cast<int>(mb.ckpts.size()) - 1; k >= 0; --k) {
            const long long n0 = mb.ckpts[k].first;
            TRY(back_steps(n - n0));
            n = n0;
            // re-anchor the reconstructed forward state on the FP64 checkpoint
            const double *ck = mb.ckpts[k].second;
            CUDA_TRY(c, adjoint_load_state(d, elem, view(), ck, ck + cells, c->stream));
        }
        if (mb.from_packet)
            CUDA_TRY(c, adjoint_start_term(d, elem, view(), mb.ckpts[0].second, c->stream));
        if (dL_dV)
            CUDA_TRY(c, cudaMemcpyAsync(dL_dV, gV, cells * 8,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        c->stream));
        if (dL_datoms) {
            const int na = static_cast<int>(mb.atoms.size() / 4);
            void *A, *part, *outA;
            TRY(alloc(mb.atoms.size() * 8, &A));
            TRY(alloc(static_cast<size_t>(na) * atom_grad_chunks() * 4 * 8, &part));
            TRY(alloc(mb.atoms.size() * 8, &outA));
            CUDA_TRY(c, cudaMemcpyAsync(A, mb.atoms.data(), mb.atoms.size() * 8,
                                        cudaMemcpyHostToDevice, c->stream));
            CUDA_TRY(c, launch_atom_gradient(d, static_cast<double *>(A), na, mb.soft_a2, mb.r_cut,
                                             static_cast<double *>(gV), static_cast<double *>(part),
                                             static_cast<double *>(outA), c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(dL_datoms, outA, mb.atoms.size() * 8,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                        c->stream));
        }
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        return TDSE_OK;
    };
    st = run();
    cleanup();
    drop_graphs();
    if (st == TDSE_OK) st = resolve_timers(c);   // the stream is synchronised
    return st;
}

tdse_status tdse_save_state(tdse_ctx *c, const char *path)
{
    if (!c || !path) return TDSE_EINVAL;
    TRY(check_usable(c));
    for (const Member &mb : c->m)
        if (!mb.have_state) return fail(c, TDSE_ESTATE, "every member needs a state to be saved");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(c, TDSE_EINVAL, "cannot open %s for writing", path);
    bool ok = put(f, kMagic, 8);
    const int B = static_cast<int>(c->m.size());
    ok = ok && put(f, &B, 1) && put(f, &c->step, 1);
    std::vector<double> host;
    for (Member &mb : c->m) {
        const size_t cells = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz;
        const size_t pix = static_cast<size_t>(mb.dev.nx) * mb.dev.ny;
        const int from = mb.from_packet, nh = static_cast<int>(mb.hist.size()),
                  na = static_cast<int>(mb.atoms.size()), nck = static_cast<int>(mb.ckpts.size());
        ok = ok && put(f, &mb.p, 1) && put(f, &from, 1) && put(f, &mb.q0, 1) &&
             put(f, &mb.soft_a2, 1) && put(f, &mb.r_cut, 1);
        ok = ok && put(f, &nh, 1) && put(f, mb.hist.data(), nh) && put(f, &na, 1) &&
             put(f, mb.atoms.data(), na);
        // raw fields: R, I (and the Kahan compensation terms), exact in FP64
        const int nf = c->precision == TDSE_FP32_KAHAN ? 4 : 2;
        void *fields[4] = {mb.dev.R[c->cur], mb.dev.I[c->cur], mb.dev.cR[c->cur], mb.dev.cI[c->cur]};
        void *tmp = nullptr;
        TRY(dalloc(c, cells * 8, &tmp));
        host.resize(cells);
        for (int k = 0; k < nf; ++k) {
            CUDA_TRY(c, launch_field_io(mb.dev, fields[k], static_cast<int>(elem_size(c->precision)),
                                        static_cast<double *>(tmp), 0, c->stream));
            CUDA_TRY(c, cudaMemcpyAsync(host.data(), tmp, cells * 8, cudaMemcpyDeviceToHost, c->stream));
            CUDA_TRY(c, cudaStreamSynchronize(c->stream));
            ok = ok && put(f, host.data(), cells);
        }
        dfree(c, tmp);
        host.resize(2 * cells);
        CUDA_TRY(c, cudaMemcpy(host.data(), mb.V64, cells * 8, cudaMemcpyDeviceToHost));
        ok = ok && put(f, host.data(), cells);
        CUDA_TRY(c, cudaMemcpy(host.data(), mb.dev.flux, pix * 8, cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(host.data() + pix, mb.dev.jlast, pix * 8, cudaMemcpyDeviceToHost));
        ok = ok && put(f, host.data(), 2 * pix) && put(f, &nck, 1);
        for (auto &ck : mb.ckpts) {
            CUDA_TRY(c, cudaMemcpy(host.data(), ck.second, 2 * cells * 8, cudaMemcpyDeviceToHost));
            ok = ok && put(f, &ck.first, 1) && put(f, host.data(), 2 * cells);
        }
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? TDSE_OK : fail(c, TDSE_EINVAL, "write to %s failed", path);
}

tdse_status tdse_load_state(tdse_ctx *c, const char *path)
{
    if (!c || !path) return TDSE_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(c, TDSE_EINVAL, "cannot open %s", path);
    auto bad = [&](const char *why) {
        fclose(f);
        return fail(c, TDSE_EINVAL, "%s: %s", path, why);
    };
    char magic[8];
    int B = 0;
    long long step = 0;
    if (!get(f, magic, 8) || memcmp(magic, kMagic, 8) != 0) return bad("not a tdse state file");
    if (!get(f, &B, 1) || B != static_cast<int>(c->m.size()) || !get(f, &step, 1))
        return bad("batch size differs");
    tdse_status st = ensure_device(c);
    if (st != TDSE_OK) {
        fclose(f);
        return st;
    }
    std::vector<double> host;
    for (Member &mb : c->m) {
        const size_t cells = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * mb.dev.nz;
        const size_t pix = static_cast<size_t>(mb.dev.nx) * mb.dev.ny;
        tdse_params p;
        int from = 0, nh = 0, na = 0, nck = 0;
        double q0 = 0, a2 = 0, rc = 0;
        if (!get(f, &p, 1) || !same_grid(p, mb.p)) return bad("parameters differ from the context's");
        if (!get(f, &from, 1) || !get(f, &q0, 1) || !get(f, &a2, 1) || !get(f, &rc, 1) ||
            !get(f, &nh, 1) || nh < 0)
            return bad("truncated");
        std::vector<double> hist(nh), atoms;
        if (!get(f, hist.data(), nh) || !get(f, &na, 1) || na < 0) return bad("truncated");
        atoms.resize(na);
        const int nf = c->precision == TDSE_FP32_KAHAN ? 4 : 2;
        host.resize((nf + 1) * cells);
        if (!get(f, atoms.data(), na) || !get(f, host.data(), (nf + 1) * cells)) return bad("truncated");
        // potential, then the raw fields into the current buffer
        void *tmp = nullptr;
        TRY(dalloc(c, (nf + 1) * cells * 8, &tmp));
        double *dv = static_cast<double *>(tmp);
        CUDA_TRY(c, cudaMemcpy(dv, host.data(), (nf + 1) * cells * 8, cudaMemcpyHostToDevice));
        TRY(potential_to_d(c, mb, dv + nf * cells));
        void *fields[4] = {mb.dev.R[c->cur], mb.dev.I[c->cur], mb.dev.cR[c->cur], mb.dev.cI[c->cur]};
        for (int k = 0; k < nf; ++k)
            CUDA_TRY(c, launch_field_io(mb.dev, fields[k], static_cast<int>(elem_size(c->precision)),
                                        dv + k * cells, 1, c->stream));
        TRY(fill_all_ghosts(c, mb, c->cur));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        dfree(c, tmp);
        host.resize(2 * pix);
        if (!get(f, host.data(), 2 * pix) || !get(f, &nck, 1) || nck < 0) return bad("truncated");
        CUDA_TRY(c, cudaMemcpy(mb.dev.flux, host.data(), pix * 8, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(mb.dev.jlast, host.data() + pix, pix * 8, cudaMemcpyHostToDevice));
        clear_checkpoints(c, mb);
        host.resize(2 * cells);
        for (int k = 0; k < nck; ++k) {
            long long s = 0;
            if (!get(f, &s, 1) || !get(f, host.data(), 2 * cells)) return bad("truncated");
            void *ck = nullptr;
            TRY(dalloc(c, 2 * cells * 8, &ck));
            CUDA_TRY(c, cudaMemcpy(ck, host.data(), 2 * cells * 8, cudaMemcpyHostToDevice));
            mb.ckpts.push_back({s, static_cast<double *>(ck)});
        }
        mb.from_packet = from != 0;
        mb.q0 = q0;
        mb.hist = hist;
        mb.atoms = atoms;
        mb.soft_a2 = a2;
        mb.r_cut = rc;
        mb.have_state = true;
    }
    fclose(f);
    c->step = step;
    for (size_t i = 0; i < c->m.size(); ++i) c->obs_slices[i].q_ref = c->m[i].q0;
    CUDA_TRY(c, cudaMemcpy(c->d_obs_slices, c->obs_slices.data(), c->obs_slices.size() * sizeof(ObsSlice),
                           cudaMemcpyHostToDevice));
    return TDSE_OK;
}

int tdse_variant_count(int precision, int tsteps) { return step_variant_count(precision, tsteps); }

tdse_status tdse_set_variant(tdse_ctx *c, int tsteps, int variant)
{
    if (!c) return TDSE_EINVAL;
    if (tsteps < 1 || tsteps > kMaxTblock || variant < 0 ||
        variant >= step_variant_count(c->precision, tsteps))
        return fail(c, TDSE_EINVAL, "no variant %d for %d fused steps", variant, tsteps);
    TRY(ensure_device(c));
    return build_plan(c, tsteps, variant);
}

tdse_status tdse_set_wait_limit(tdse_ctx *c, long long ns)
{
    if (!c) return TDSE_EINVAL;
    if (ns < 0) return fail(c, TDSE_EINVAL, "negative wait limit");
    c->wait_ns = static_cast<unsigned long long>(ns);
    drop_graphs(c);   // captured launches carry the limit as an argument
    return TDSE_OK;
}

tdse_status tdse_set_adjoint_fused(tdse_ctx *c, int enable)
{
    if (!c) return TDSE_EINVAL;
    c->adjoint_fused = enable != 0;
    return TDSE_OK;
}

tdse_status tdse_set_chunk(tdse_ctx *c, int tsteps, int planes)
{
    if (!c) return TDSE_EINVAL;
    if (tsteps < 1 || tsteps > kMaxTblock || step_variant_count(c->precision, tsteps) == 0)
        return fail(c, TDSE_EINVAL, "no kernel variants for %d fused steps", tsteps);
    if (planes < 0) return fail(c, TDSE_EINVAL, "negative chunk length");
    TRY(ensure_device(c));
    c->plans[tsteps].chunk_request = planes;
    return build_plan(c, tsteps, c->plans[tsteps].variant);
}

tdse_status tdse_set_graphs(tdse_ctx *c, int enable)
{
    if (!c) return TDSE_EINVAL;
    c->graphs = enable != 0;
    return TDSE_OK;
}

tdse_status tdse_get_tuning(tdse_ctx *c, tdse_tuning *out)
{
    if (!c || !out) return TDSE_EINVAL;
    memset(out, 0, sizeof *out);
    out->tblock = c->tblock;
    for (int T = 1; T <= kMaxTblock; ++T) {
        if (step_variant_count(c->precision, T) == 0) continue;
        out->variant[T] = c->plans[T].variant;
        out->chunk[T] = c->plans[T].chunk;
        out->ms_per_step[T] = c->tuned_ms_per_step[T];
        const char *n = step_variant_name(c->precision, T, c->plans[T].variant);
        if (n) snprintf(out->name[T], sizeof out->name[T], "%s", n);
    }
    return TDSE_OK;
}

tdse_status tdse_autotune(tdse_ctx *c, int launches)
{
    if (!c || launches < 1) return TDSE_EINVAL;
    TRY(check_usable(c));
    TRY(ensure_device(c));
    // save what the trial launches overwrite
    const size_t es = elem_size(c->precision);
    const int nf = c->precision == TDSE_FP32_KAHAN ? 4 : 2;
    std::vector<void *> saved;
    auto field = [&](Member &mb, int f, int buf) -> void * {
        return f == 0 ? mb.dev.R[buf] : f == 1 ? mb.dev.I[buf] : f == 2 ? mb.dev.cR[buf] : mb.dev.cI[buf];
    };
    for (Member &mb : c->m) {
        const size_t fbytes = static_cast<size_t>(mb.dev.plane) * mb.dev.nz * es;
        const size_t pbytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * sizeof(double);
        for (int f = 0; f < nf; ++f) {
            void *p;
            TRY(dalloc(c, fbytes, &p));
            CUDA_TRY(c, cudaMemcpyAsync(p, field(mb, f, c->cur), fbytes, cudaMemcpyDeviceToDevice, c->stream));
            saved.push_back(p);
        }
        for (double *src : {mb.dev.flux, mb.dev.jlast}) {
            void *p;
            TRY(dalloc(c, pbytes, &p));
            CUDA_TRY(c, cudaMemcpyAsync(p, src, pbytes, cudaMemcpyDeviceToDevice, c->stream));
            saved.push_back(p);
        }
    }
    const int cur0 = c->cur;
    const long long step0 = c->step;
    const bool prof0 = c->profiling;
    const int tb0 = c->tblock;
    c->profiling = false;
    cudaEvent_t e0, e1;
    CUDA_TRY(c, cudaEventCreate(&e0));
    CUDA_TRY(c, cudaEventCreate(&e1));
    tdse_status st = TDSE_OK;
    for (int T = 1; T <= kMaxTblock && st == TDSE_OK; ++T) {
        if (step_variant_count(c->precision, T) == 0) continue;
        c->tblock = T;
        double best = 1e300;
        int bestv = 0;
        // ms per step of the plan as built (one warm-up launch, then `launches`)
        auto trial = [&](double *per_step) -> tdse_status {
            TRY(launch_fused(c, T));
            cudaEventRecord(e0, c->stream);
            for (int l = 0; l < launches; ++l) TRY(launch_fused(c, T));
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) return fail(c, TDSE_ECUDA, "autotune launch failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            *per_step = ms / (launches * T);
            return TDSE_OK;
        };
        StepPlan &pl = c->plans[T];
        const int request = pl.chunk_request;   // a chunk fixed by tdse_set_chunk stays
        // Every variant at z-chunks of 1, 0.7, 0.5, 0.35 and 0.2 of the makespan
        // model's length for it, then the best pair at 0.85 .. 1.15 of its chunk
        // (in steps of 0.05).
        // Shorter chunks cost pipeline fill but keep neighbouring tiles close in z
        // (their shared halo rows are still in L2), and the number of work items
        // against the number of CTAs decides how full the last wave is; the model
        // counts only the fill and the waves, so both are measured.
        int best_req = request;
        std::vector<int> tried;
        struct Cand {
            double ms;
            int v, req;
        };
        std::vector<Cand> cands;   // every (variant, chunk) timed, with its best time
        auto try_chunk = [&](int v, int req) -> tdse_status {
            double per_step = 0.0;
            pl.chunk_request = req;
            TRY(build_plan(c, T, v));
            TRY(trial(&per_step));
            if (per_step < best) {
                best = per_step;
                bestv = v;
                best_req = req;
            }
            cands.push_back(Cand{per_step, v, req});
            return TDSE_OK;
        };
        for (int v = 0; v < step_variant_count(c->precision, T) && st == TDSE_OK; ++v) {
            pl.chunk_request = request;
            if ((st = build_plan(c, T, v)) != TDSE_OK) break;
            const int model = pl.chunk;
            tried.clear();
            for (int frac20 : {20, 14, 10, 7, 4}) {
                if (request > 0 && frac20 != 20) break;
                const int L = frac20 == 20 ? request : model * frac20 / 20;
                if (frac20 != 20 && (L < 16 || std::find(tried.begin(), tried.end(), L) != tried.end())) continue;
                tried.push_back(frac20 == 20 ? model : L);
                if ((st = try_chunk(v, L)) != TDSE_OK) break;
            }
        }
        if (st == TDSE_OK && request == 0) {
            pl.chunk_request = best_req;
            if ((st = build_plan(c, T, bestv)) == TDSE_OK) {   // best_req as built: its chunk
                const int L0 = pl.chunk;
                for (int frac20 : {17, 18, 19, 21, 22, 23}) {
                    const int L = L0 * frac20 / 20;
                    if (L < 16 || L == L0) continue;
                    if ((st = try_chunk(bestv, L)) != TDSE_OK) break;
                }
            }
        }
        // One timing per candidate can rank two candidates a few per cent apart in
        // the wrong order, so the fastest four are timed twice more, in turn, and
        // each keeps its best time.
        if (st == TDSE_OK && cands.size() > 1) {
            std::stable_sort(cands.begin(), cands.end(), [](const Cand &a, const Cand &b) { return a.ms < b.ms; });
            std::vector<Cand> top;
            for (const Cand &k : cands) {
                bool dup = false;
                for (const Cand &t : top) dup |= t.v == k.v && t.req == k.req;
                if (!dup) top.push_back(k);
                if (top.size() == 4) break;
            }
            for (int rep = 0; rep < 2 && st == TDSE_OK; ++rep)
                for (Cand &k : top) {
                    double per_step = 0.0;
                    pl.chunk_request = k.req;
                    if ((st = build_plan(c, T, k.v)) != TDSE_OK || (st = trial(&per_step)) != TDSE_OK) break;
                    k.ms = std::min(k.ms, per_step);
                }
            if (st == TDSE_OK) {
                const Cand *b = &top[0];
                for (const Cand &k : top)
                    if (k.ms < b->ms) b = &k;
                best = b->ms;
                bestv = b->v;
                best_req = b->req;
            }
        }
        pl.chunk_request = best_req;
        if (st == TDSE_OK) st = build_plan(c, T, bestv);
        c->tuned_ms_per_step[T] = best;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->tblock = tb0;
    if (st == TDSE_OK && c->tblock_auto) {   // the depth with the lowest time per step
        for (int T = 1; T <= kMaxTblock; ++T)
            if (c->tuned_ms_per_step[T] > 0 && c->tuned_ms_per_step[T] < c->tuned_ms_per_step[c->tblock])
                c->tblock = T;
    }
    // restore the state, the flux integral and the counters
    size_t k = 0;
    for (Member &mb : c->m) {
        const size_t fbytes = static_cast<size_t>(mb.dev.plane) * mb.dev.nz * es;
        const size_t pbytes = static_cast<size_t>(mb.dev.nx) * mb.dev.ny * sizeof(double);
        for (int f = 0; f < nf; ++f)
            cudaMemcpyAsync(field(mb, f, cur0), saved[k++], fbytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(mb.dev.flux, saved[k++], pbytes, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(mb.dev.jlast, saved[k++], pbytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (void *p : saved) dfree(c, p);
    c->cur = cur0;
    c->step = step0;
    c->profiling = prof0;
    c->prof = tdse_profile{};
    return st;
}

tdse_status tdse_set_profiling(tdse_ctx *c, int enable)
{
    if (!c) return TDSE_EINVAL;
    c->profiling = enable != 0;
    c->prof = tdse_profile{};
    return TDSE_OK;
}

tdse_status tdse_get_profile(tdse_ctx *c, tdse_profile *out)
{
    if (!c || !out) return TDSE_EINVAL;
    *out = c->prof;
    return TDSE_OK;
}

tdse_status tdse_destroy(tdse_ctx *c)
{
    if (!c) return TDSE_OK;
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->event_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->status_ev)
        if (e) cudaEventDestroy(e);
    if (c->h_status) cudaFreeHost(c->h_status);
    drop_graphs(c);
    if (c->gstream) {
        cudaStreamSynchronize(c->gstream);
        cudaStreamDestroy(c->gstream);
        cudaEventDestroy(c->gev[0]);
        cudaEventDestroy(c->gev[1]);
    }
    std::vector<void *> all = c->allocations;
    for (void *p : all) dfree(c, p);
    delete c;
    return TDSE_OK;
}

}  // extern "C"
