// Detector-plane data (arXiv 2401.07416, Sec. 2.3 and Sec. 3.2): the density frames
// of Eq. 15 and the trajectory dissimilarity of Eq. 16.
//
// Frames: rho[y][x] = R^n^2 + I^{n-1/2}^2 on plane det_k (FP64 from the stored
// fields, Kahan value minus compensation).
//
// Dissimilarity: for the frames m in the window [t0, t1] and every pair k <= j,
//   S[m][k][j] = sum_p (rho_k[m][p] - rho_j[m][p])^2            (pair_sq_kernel)
//   d[k][j] = d[j][k] = sum_m w_m sqrt(dA S[m][k][j]) / (t1 - t0) (pair_time_kernel)
// with trapezoidal weights w_m on the window's frame times.  pair_sq_kernel is a
// tiled pairwise-distance kernel: a block owns a 32 x 32 tile of (k, j) pairs of
// one frame (upper-triangle tiles only), stages 32-pixel chunks of the 32 + 32
// trajectories in shared memory and each thread accumulates a 2 x 2 sub-tile in
// FP64, the pixel sum in a fixed order (reproducible).
#include <cmath>
#include <vector>

#include "tdse.h"
#include "tdse_internal.cuh"

namespace tdse {
namespace {

constexpr int kTile = 32;      // trajectories per tile side
constexpr int kChunk = 32;     // pixels per shared-memory chunk

template <typename Real>
__global__ void frame_kernel(MemberDev m, int buf, int kahan, double *__restrict__ out)
{
    const Real *R = reinterpret_cast<const Real *>(m.R[buf]);
    const Real *I = reinterpret_cast<const Real *>(m.I[buf]);
    const Real *cR = kahan ? reinterpret_cast<const Real *>(m.cR[buf]) : nullptr;
    const Real *cI = kahan ? reinterpret_cast<const Real *>(m.cI[buf]) : nullptr;
    const int npix = m.nx * m.ny;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < npix; t += gridDim.x * blockDim.x) {
        const int x = t % m.nx, y = t / m.nx;
        const long long o = static_cast<long long>(m.det_k) * m.plane +
                            static_cast<long long>(y + m.G) * m.pitch + (x + m.G);
        double r = static_cast<double>(R[o]), i = static_cast<double>(I[o]);
        if (kahan) {
            r -= static_cast<double>(cR[o]);
            i -= static_cast<double>(cI[o]);
        }
        out[t] = r * r + i * i;
    }
}

// S[mi][k][j] for the window frame frame_idx[mi], tile (blockIdx.y, blockIdx.x), k <= j tiles.
__global__ void __launch_bounds__(256)
    pair_sq_kernel(const double *__restrict__ F, int K, int M, long long P,
                   const int *__restrict__ frame_idx, double *__restrict__ S)
{
    const int bk = blockIdx.y, bj = blockIdx.x;
    if (bk > bj) return;
    __shared__ double A[kTile][kChunk + 1];
    __shared__ double B[kTile][kChunk + 1];
    const int mi = blockIdx.z;
    const int m = frame_idx[mi];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int k0 = bk * kTile, j0 = bj * kTile;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    for (long long p0 = 0; p0 < P; p0 += kChunk) {
        for (int e = threadIdx.x; e < kTile * kChunk; e += blockDim.x) {
            const int r = e / kChunk, cc = e % kChunk;
            const long long p = p0 + cc;
            const int k = k0 + r, j = j0 + r;
            A[r][cc] = (k < K && p < P) ? F[(static_cast<long long>(k) * M + m) * P + p] : 0.0;
            B[r][cc] = (j < K && p < P) ? F[(static_cast<long long>(j) * M + m) * P + p] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int cc = 0; cc < kChunk; ++cc) {
            const double a0 = A[2 * ty][cc], a1 = A[2 * ty + 1][cc];
            const double b0 = B[2 * tx][cc], b1 = B[2 * tx + 1][cc];
            const double d00 = a0 - b0, d01 = a0 - b1, d10 = a1 - b0, d11 = a1 - b1;
            acc[0][0] = fma(d00, d00, acc[0][0]);
            acc[0][1] = fma(d01, d01, acc[0][1]);
            acc[1][0] = fma(d10, d10, acc[1][0]);
            acc[1][1] = fma(d11, d11, acc[1][1]);
        }
        __syncthreads();
    }
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            const int k = k0 + 2 * ty + a, j = j0 + 2 * tx + b;
            if (k < K && j < K) S[(static_cast<long long>(mi) * K + k) * K + j] = acc[a][b];
        }
}

__global__ void pair_time_kernel(const double *__restrict__ S, int K, int Mw,
                                 const double *__restrict__ w, double dA, double inv_span,
                                 double *__restrict__ d)
{
    const long long n = static_cast<long long>(K) * K;
    for (long long e = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; e < n;
         e += static_cast<long long>(gridDim.x) * blockDim.x) {
        const int k = static_cast<int>(e / K), j = static_cast<int>(e % K);
        if (k > j) continue;
        double s = 0.0;
        if (k != j)
            for (int mi = 0; mi < Mw; ++mi)
                s += w[mi] * sqrt(dA * S[(static_cast<long long>(mi) * K + k) * K + j]);
        s *= inv_span;
        d[static_cast<long long>(k) * K + j] = s;
        d[static_cast<long long>(j) * K + k] = s;
    }
}

}  // namespace

cudaError_t launch_frame(const MemberDev &m, int precision, int buf, double *out, cudaStream_t s)
{
    const int npix = m.nx * m.ny;
    const int grid = (npix + 255) / 256;
    if (precision == 0)
        frame_kernel<double><<<grid, 256, 0, s>>>(m, buf, 0, out);
    else
        frame_kernel<float><<<grid, 256, 0, s>>>(m, buf, precision == 2, out);
    return cudaGetLastError();
}

}  // namespace tdse

using namespace tdse;

extern "C" TDSE_API tdse_status tdse_dissimilarity(const double *frames, int K, int M, long long P,
                                                   const double *t, double t0, double t1,
                                                   double dA, double *d, int on_device,
                                                   void *stream)
{
    if (!frames || !t || !d || K < 1 || M < 1 || P < 1 || !(dA > 0.0) || !(t1 > t0))
        return TDSE_EINVAL;
    // window frames and trapezoidal weights (t is a host array)
    std::vector<int> idx;
    for (int m = 0; m < M; ++m)
        if (t[m] >= t0 && t[m] <= t1) idx.push_back(m);
    if (idx.empty()) return TDSE_EINVAL;
    std::vector<double> w(idx.size(), 0.0);
    if (idx.size() == 1) {
        w[0] = t1 - t0;
    } else {
        for (size_t a = 0; a + 1 < idx.size(); ++a) {
            const double half = 0.5 * (t[idx[a + 1]] - t[idx[a]]);
            w[a] += half;
            w[a + 1] += half;
        }
    }
    const int Mw = static_cast<int>(idx.size());
    if (Mw > 65535) return TDSE_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t fbytes = static_cast<size_t>(K) * M * P * sizeof(double);
    const size_t sbytes = static_cast<size_t>(Mw) * K * K * sizeof(double);
    const size_t dbytes = static_cast<size_t>(K) * K * sizeof(double);
    void *dF = nullptr, *dS = nullptr, *dW = nullptr, *dI = nullptr, *dD = nullptr;
    auto release = [&]() {
        if (!on_device && dF) cudaFreeAsync(dF, s);
        if (!on_device && dD) cudaFreeAsync(dD, s);
        if (dS) cudaFreeAsync(dS, s);
        if (dW) cudaFreeAsync(dW, s);
        if (dI) cudaFreeAsync(dI, s);
        cudaStreamSynchronize(s);
    };
    auto oom = [&](cudaError_t e) { return e == cudaErrorMemoryAllocation ? TDSE_ENOMEM : TDSE_ECUDA; };
    cudaError_t e = cudaSuccess;
    if (on_device) {
        dF = const_cast<double *>(frames);
        dD = d;
    } else {
        if ((e = cudaMallocAsync(&dF, fbytes, s)) != cudaSuccess ||
            (e = cudaMallocAsync(&dD, dbytes, s)) != cudaSuccess) {
            release();
            return oom(e);
        }
    }
    if ((e = cudaMallocAsync(&dS, sbytes, s)) != cudaSuccess ||
        (e = cudaMallocAsync(&dW, Mw * sizeof(double), s)) != cudaSuccess ||
        (e = cudaMallocAsync(&dI, Mw * sizeof(int), s)) != cudaSuccess) {
        release();
        return oom(e);
    }
    tdse_status st = TDSE_OK;
    do {
        if (!on_device &&
            cudaMemcpyAsync(dF, frames, fbytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = TDSE_ECUDA;
            break;
        }
        if (cudaMemcpyAsync(dW, w.data(), Mw * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(dI, idx.data(), Mw * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = TDSE_ECUDA;
            break;
        }
        const int tiles = (K + kTile - 1) / kTile;
        pair_sq_kernel<<<dim3(tiles, tiles, Mw), 256, 0, s>>>(static_cast<const double *>(dF), K, M,
                                                               P, static_cast<int *>(dI),
                                                               static_cast<double *>(dS));
        const long long pairs = static_cast<long long>(K) * K;
        const int grid = static_cast<int>(std::min<long long>((pairs + 255) / 256, 152LL * 16));
        pair_time_kernel<<<grid, 256, 0, s>>>(static_cast<double *>(dS), K, Mw,
                                              static_cast<double *>(dW), dA, 1.0 / (t1 - t0),
                                              static_cast<double *>(dD));
        if (cudaGetLastError() != cudaSuccess) {
            st = TDSE_ECUDA;
            break;
        }
        if (!on_device &&
            cudaMemcpyAsync(d, dD, dbytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            st = TDSE_ECUDA;
            break;
        }
    } while (false);
    release();
    if (st == TDSE_OK && cudaStreamSynchronize(s) != cudaSuccess) st = TDSE_ECUDA;
    return st;
}
