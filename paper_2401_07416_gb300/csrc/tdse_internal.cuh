// Internal declarations shared by the translation units of libtdse.
//
// Device data layout of one member (all fields of the context's precision Real):
//   padded planes of (nx + 2G) x (ny + 2G) nodes with ghost width G on x and y;
//   row pitch `pitch` elements (a multiple of 16 bytes), `prow` = ny + 2G rows,
//   nz planes; element (x, y, z) with unpadded x in [-G, nx+G) lives at
//   ((z * prow) + (y + G)) * pitch + (x + G).
//   Periodic axes keep copies of the opposite boundary strips in their ghost
//   zones (refreshed by every kernel that writes the field); walled axes keep
//   zeros there.  The fused step reads whole tiles with TMA and never wraps
//   indices in x or y.
// Fields: R[2], I[2] (ping-pong: each step launch reads one and writes the other),
//   cR[2], cI[2] (Kahan compensation, FP32_KAHAN only), d (the diagonal of the
//   operator A: d = -2 (c_x + c_y + c_z) - c_v V), flux and jlast (FP64 [ny][nx]),
//   mask[nz] (Real).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "tdse.h"

namespace tdse {

constexpr int kGhost = 8;          // ghost width on x and y (supports up to 4 fused steps)
constexpr int kMaxTblock = TDSE_MAX_TBLOCK;   // largest number of steps fused per launch

struct alignas(128) MemberDev {
    CUtensorMap tm_R[2], tm_I[2], tm_cR[2], tm_cI[2], tm_d;
    void *R[2];
    void *I[2];
    void *cR[2];
    void *cI[2];
    void *d;
    void *mask;            // Real[nz]
    double *flux;          // [ny][nx], time-integrated flux
    double *jlast;         // [ny][nx], flux of the last step
    long long plane;       // elements per padded plane = pitch * prow
    int nx, ny, nz, G, pitch, prow;
    int per_x, per_y, per_z, det_k;
    int mask_lo, mask_hi;     // absorbing planes at the z ends
    double cx, cy, cz, cv, cj, dt;
    double hx, hy, hz, hbar;
};

// Work decomposition of one fused-step launch configuration over all members:
// member m owns items [item_begin[m], item_begin[m+1]); item i of member m is
// tile (i % tiles_x, (i / tiles_x) % tiles_y) of z-chunk i / (tiles_x tiles_y).
struct WorkDev {
    int nmembers;
    int total;
    int item_begin[257];
    int tiles_x[256];
    int tiles_y[256];
    int chunk[256];        // z planes per chunk (last chunk may be shorter)
};

struct StepLaunch {
    const MemberDev *members;
    const WorkDev *work;
    int *counter;          // dynamic work counter, zeroed before the launch
    int *status;           // error word (bit 0: a wait for a tile's data expired; bit 2: a
                           // CTA left with a load in flight after its drain wait expired)
    int in_buf;            // ping-pong index read by this launch
    unsigned long long wait_ns;   // limit of each wait for a tile's data (0: test once)
    int grid, block;
    size_t smem;
    cudaStream_t stream;
};

// Launch configuration of a fused step: precision, fused steps and Kahan.
struct StepConfig {
    int tile_x, tile_y;    // output tile (x, y)
    int box_x, box_y;      // TMA box (region) loaded per plane
    int threads;
    size_t smem;
    int ctas_per_sm;
};

// step_kernels.cu: kernel variants (tile shape, prefetch depth) per precision
// and number of fused steps; variant 0 is the default.
int step_variant_count(int precision, int tsteps);
const char *step_variant_name(int precision, int tsteps, int variant);
bool step_config(int precision, int tsteps, int variant, StepConfig *cfg);
cudaError_t launch_step(int precision, int tsteps, int variant, const StepLaunch &L);

// aux_kernels.cu
cudaError_t launch_fill_ghosts(const MemberDev &m, void *field, int elem, cudaStream_t s);
// V[nz][ny][nx] (FP64) from n atoms [n][4]; `scratch` holds atom_cell_bytes(n).
// precision 0 evaluates every term in FP64, otherwise the profile in FP32.
cudaError_t launch_potential_atoms(const MemberDev &m, const double *atoms, int n, double a2,
                                   double rc, double *V, void *scratch, int precision,
                                   cudaStream_t s);
size_t atom_cell_bytes(int n);
// d (padded, Real) from V (unpadded FP64, NULL: V = 0); V copied into V64
cudaError_t launch_build_d(const MemberDev &m, int elem, const double *V, double *V64,
                           cudaStream_t s);
// Eq. 3 packet and the half-step start I^{-1/2} = Im psi0 - A[Re psi0]/2 written straight
// into the state (scratch: packet_scratch_bytes, device memory).
size_t packet_scratch_bytes(const MemberDev &m);
cudaError_t launch_packet_start(const MemberDev &m, const double *V64, const double *r0,
                                const double *sigma, const double *k0, void *scratch,
                                int precision, int buf, cudaStream_t s);
cudaError_t launch_set_state(const MemberDev &m, const double *R64, const double *I64,
                             int precision, int buf, cudaStream_t s);
// Trilinear interpolation of a periodic cell potential onto the grid (FP64, unpadded;
// scratch: interp_scratch_bytes, device memory).
size_t interp_scratch_bytes(const MemberDev &m);
cudaError_t launch_interp(const MemberDev &m, double hx, double hy, double hz, const double *Vc,
                          int cnx, int cny, int cnz, const double L[3], const double o[3],
                          void *scratch, double *V, cudaStream_t s);
// Eq. 15 density of plane det_k at the current time level into out[ny][nx] (FP64).
cudaError_t launch_frame(const MemberDev &m, int precision, int buf, double *out, cudaStream_t s);
cudaError_t launch_get_state(const MemberDev &m, double *R64, double *I64, int precision,
                             int buf, cudaStream_t s);
// copy the interior of one padded field out to (to_field = 0) or in from an
// unpadded FP64 array (exact for values representable in the field's type)
cudaError_t launch_field_io(const MemberDev &m, void *field, int elem, double *array, int to_field,
                            cudaStream_t s);
// record[0..5] = {step, Q, norm_paper, energy, flux_last, flux_integrated}.  Sets status bit 1 if Q is
// not finite or exceeds (1 + 1e-3) q_ref (q_ref <= 0: no growth check).
cudaError_t launch_observables(const MemberDev &m, int precision, int buf, double *partials,
                               double *record, int *status, double q_ref, long long step,
                               cudaStream_t s);
// One member's share of a batched reduction launch (observables_batch_kernel).
struct ObsSlice {
    int block_begin;       // its first block in the launch
    int nparts;            // its blocks (as in a launch of its own)
    int zch;               // z planes per work item
    double q_ref;          // Q of its first observation (<= 0: no growth check)
};
// Blocks and z-chunk of one member's reduction (the same in both launch forms).
void observables_shape(const MemberDev &m, int precision, int *nparts, int *zch);
// Every member's reduction in two launches; member i's record goes to
// records + i * rec_stride.  Bitwise the same records as launch_observables per member.
cudaError_t launch_observables_batch(const MemberDev *members, const ObsSlice *slices, int nmembers,
                                     int total_blocks, int precision, int buf, double *partials,
                                     double *records, long long rec_stride, int *status, long long step,
                                     cudaStream_t s);
constexpr int kObsParts = 1216;     // fixed block count: the reduction order never changes
constexpr int kObsZ = 64;           // largest z-chunk of an observables work item
constexpr int kObsZmin = 16;        // smallest z-chunk of an observables work item
constexpr int kObsThreads = 256;    // observables block size
constexpr int kObsBlocksPerSM = 2;  // resident observables blocks per SM (up to 128 registers per thread)
constexpr int kObsPartialsPerBlock = 5;   // Q, paper norm, energy, flux (last step, integrated)

// adjoint_kernels.cu: working arrays of one backward sweep (unpadded, Real of the
// context for R, I, P, Q; FP64 for the rest).
struct AdjointBuffers {
    void *R, *I;          // forward state being reconstructed: R^n, I^{n-1/2}
    void *P, *Q;          // their adjoints
    void *R2, *I2, *P2, *Q2;   // second set for the fused step, which reads one set and
                               // writes the other (NULL: three passes in place)
    double *gV;           // dL/dV accumulator
    double *w;            // dL/dF * dt * cj per detector pixel
    const void *Minv;     // reciprocal of the absorbing factor per plane (the context's
                          // number format, like MemberDev::mask)
    void *Ist;            // It of the two detector planes (2 nx ny values, that format)
    const double *V;      // potential (FP64)
};
// One backward step.  With a second buffer set, one fused z-march that reads (R, I, P,
// Q) and writes (R2, I2, P2, Q2), after which the caller swaps the two sets; without,
// three passes in place.
cudaError_t adjoint_backward_step(const MemberDev &m, int elem, const AdjointBuffers &b,
                                  cudaStream_t s);
cudaError_t adjoint_start_term(const MemberDev &m, int elem, const AdjointBuffers &b,
                               const double *R0, cudaStream_t s);
cudaError_t adjoint_load_state(const MemberDev &m, int elem, const AdjointBuffers &b,
                               const double *R64, const double *I64, cudaStream_t s);
cudaError_t adjoint_flux_weights(const MemberDev &m, const double *gF, double *w, cudaStream_t s);
int atom_grad_chunks();
cudaError_t launch_atom_gradient(const MemberDev &m, const double *atoms, int natoms, double a2,
                                 double rc, const double *gV, double *partial, double *out,
                                 cudaStream_t s);

}  // namespace tdse
