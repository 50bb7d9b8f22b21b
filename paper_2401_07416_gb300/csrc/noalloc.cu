// Observables of an FP64 state computed without allocating device memory.
//
// tdse_observables needs a context, and a context allocates its buffers.  Some
// callers cannot allocate: a host program whose device memory is entirely owned
// by another allocator (a framework's pool or a fixed arena it must not bypass),
// or code running where a cudaMalloc would implicitly synchronise the device and
// stall other work.  tdse_observables_static serves them: the caller passes the
// state and the potential already on the device, and the reduction's scratch is
// the file-scope array below, which every GPU that loads this library keeps
// until the process exits.
#include <mutex>

#include "tdse.h"

namespace {

constexpr int kMaxPlanes = 8192;       // largest nz accepted
constexpr int kMaxDevices = 64;
constexpr int kThreads = 256;

// Per-plane partial sums (Q, paper norm, energy numerator, unused) followed by the
// final three results: (kMaxPlanes + 1) * 4 doubles = 256 KiB + 32 bytes.
static __device__ __align__(256) double g_scratch[(kMaxPlanes + 1) * 4];

std::mutex g_mutex;
double *g_scratch_addr[kMaxDevices] = {};

struct Geometry {
    int nx, ny, nz;
    int per[3];
    double cx, cy, cz, cv, h3, hbar, dt;
};

__device__ __forceinline__ double at(const double *f, const Geometry &g, int x, int y, int z)
{
    if (x < 0 || x >= g.nx) {
        if (!g.per[0]) return 0.0;
        x = (x % g.nx + g.nx) % g.nx;
    }
    if (y < 0 || y >= g.ny) {
        if (!g.per[1]) return 0.0;
        y = (y % g.ny + g.ny) % g.ny;
    }
    if (z < 0 || z >= g.nz) {
        if (!g.per[2]) return 0.0;
        z = (z % g.nz + g.nz) % g.nz;
    }
    return f[(static_cast<long long>(z) * g.ny + y) * g.nx + x];
}

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < blockDim.x / 32; ++w) s += sh[w];
    return s;
}

// One block per z plane: sums of R.R + I+.I, R^2 + I^2 and R.AR + I+.AI with
// I+ = I + A R, A f = cx(f[x+1] + f[x-1]) + cy(..) + cz(..) + (-2(cx+cy+cz) - cv V) f.
__global__ void plane_sums_kernel(const double *__restrict__ R, const double *__restrict__ I,
                                  const double *__restrict__ V, Geometry g, double *scratch)
{
    __shared__ double sh[kThreads / 32];
    const int z = blockIdx.x;
    const int n = g.nx * g.ny;
    const double c0 = -2.0 * (g.cx + g.cy + g.cz);
    double q = 0.0, pn = 0.0, e = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        const int x = t % g.nx, y = t / g.nx;
        const long long o = static_cast<long long>(z) * n + t;
        const double d = c0 - g.cv * (V ? V[o] : 0.0);
        const double r0 = R[o], i0 = I[o];
        const double ar = g.cx * (at(R, g, x + 1, y, z) + at(R, g, x - 1, y, z)) +
                          g.cy * (at(R, g, x, y + 1, z) + at(R, g, x, y - 1, z)) +
                          g.cz * (at(R, g, x, y, z + 1) + at(R, g, x, y, z - 1)) + d * r0;
        const double ai = g.cx * (at(I, g, x + 1, y, z) + at(I, g, x - 1, y, z)) +
                          g.cy * (at(I, g, x, y + 1, z) + at(I, g, x, y - 1, z)) +
                          g.cz * (at(I, g, x, y, z + 1) + at(I, g, x, y, z - 1)) + d * i0;
        const double ip = i0 + ar;
        q += r0 * r0 + ip * i0;
        pn += r0 * r0 + i0 * i0;
        e += r0 * ar + ip * ai;
    }
    q = block_sum(q, sh);
    pn = block_sum(pn, sh);
    e = block_sum(e, sh);
    if (threadIdx.x == 0) {
        scratch[4 * z + 0] = q;
        scratch[4 * z + 1] = pn;
        scratch[4 * z + 2] = e;
    }
}

// Sums the nz plane partials in plane order into the result slot.
__global__ void finalize_kernel(Geometry g, double *scratch)
{
    __shared__ double sh[kThreads / 32];
    double q = 0.0, pn = 0.0, e = 0.0;
    for (int z = threadIdx.x; z < g.nz; z += blockDim.x) {
        q += scratch[4 * z + 0];
        pn += scratch[4 * z + 1];
        e += scratch[4 * z + 2];
    }
    q = block_sum(q, sh);
    pn = block_sum(pn, sh);
    e = block_sum(e, sh);
    if (threadIdx.x == 0) {
        double *res = scratch + 4 * kMaxPlanes;
        res[0] = q * g.h3;
        res[1] = pn * g.h3;
        res[2] = -(g.hbar / g.dt) * e / q;
    }
}

// Device address of g_scratch on the current device, looked up once per device.
cudaError_t scratch_address(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" tdse_status tdse_observables_static(const tdse_params *p, const double *R,
                                               const double *I, const double *V, double out[3],
                                               void *stream)
{
    if (!p || !R || !I || !out) return TDSE_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->nz > kMaxPlanes) return TDSE_EINVAL;
    if (static_cast<long long>(p->nx) * p->ny > (1LL << 30)) return TDSE_EINVAL;   // 32-bit plane index
    if (!(p->hx > 0 && p->hy > 0 && p->hz > 0)) return TDSE_EINVAL;
    for (int a = 0; a < 3; ++a)   // the same boundary flags tdse_create accepts
        if (p->bc[a] != TDSE_BC_PERIODIC && p->bc[a] != TDSE_BC_DIRICHLET) return TDSE_EINVAL;
    const double hbar = p->hbar > 0 ? p->hbar : 1.0;
    const double mass = p->mass > 0 ? p->mass : 1.0;
    double dt = p->dt;
    if (dt <= 0) {
        double h = p->hx < p->hy ? p->hx : p->hy;
        h = h < p->hz ? h : p->hz;
        dt = mass / (5.0 * hbar) * h * h;
    }
    Geometry g;
    g.nx = p->nx;
    g.ny = p->ny;
    g.nz = p->nz;
    for (int a = 0; a < 3; ++a) g.per[a] = p->bc[a] == TDSE_BC_PERIODIC;
    g.cx = hbar * dt / (2.0 * mass * p->hx * p->hx);
    g.cy = hbar * dt / (2.0 * mass * p->hy * p->hy);
    g.cz = hbar * dt / (2.0 * mass * p->hz * p->hz);
    g.cv = dt / hbar;
    g.h3 = p->hx * p->hy * p->hz;
    g.hbar = hbar;
    g.dt = dt;
    double *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return TDSE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // launched through cudaLaunchKernel, whose status is this launch's own (an
    // error left by unrelated earlier work is neither reported nor cleared here)
    void *sum_args[] = {&R, &I, &V, &g, &scratch};
    if (cudaLaunchKernel(reinterpret_cast<const void *>(&plane_sums_kernel), dim3(g.nz), dim3(kThreads),
                         sum_args, 0, s) != cudaSuccess)
        return TDSE_ECUDA;
    void *fin_args[] = {&g, &scratch};
    if (cudaLaunchKernel(reinterpret_cast<const void *>(&finalize_kernel), dim3(1), dim3(kThreads),
                         fin_args, 0, s) != cudaSuccess)
        return TDSE_ECUDA;
    if (cudaMemcpyAsync(out, scratch + 4 * kMaxPlanes, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                        s) != cudaSuccess)
        return TDSE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return TDSE_ECUDA;
    return TDSE_OK;
}
