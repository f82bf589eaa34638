// lbm_internal.h -- host-side interface between the C ABI (lbm_api.cu) and the
// per-precision kernel translation units (lbm_f64.cu, lbm_f32.cu, ...).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_device.cuh"

namespace lbm {

struct ModesArgs {
    int32_t n_sections, n_rings, n_theta, n_modes;
    double r_over_R[16];
};

// Launch shapes of the step kernel ("variants"): threads per block, the number of
// resident blocks per SM the register budget is cut for, the planes each thread takes
// (zc), whether it is the software-pipelined persistent kernel (shapes 4 and 5, F32
// storage only) and whether it is the persistent kernel whose loads are staged in shared
// memory by bulk copies (shapes 11 and 12, compact pipe layouts, every storage; staged =
// index into STAGED_SHAPES + 1).  FP64 storage has shape 0 (256 x 2) and the staged ones.
struct StepShape { int threads, min_blocks, zc, pipelined, staged; };
constexpr StepShape STEP_SHAPES[13] = {{256, 4, 1, 0, 0}, {256, 3, 1, 0, 0}, {128, 8, 1, 0, 0}, {512, 2, 1, 0, 0},
                                       {256, 3, 1, 1, 0}, {128, 6, 1, 1, 0}, {128, 8, 2, 0, 0}, {128, 8, 4, 0, 0},
                                       {256, 4, 2, 0, 0}, {128, 7, 2, 0, 0}, {128, 6, 2, 0, 0}, {992, 1, 1, 0, 1},
                                       {512, 1, 1, 0, 2}};
constexpr StepShape STEP_SHAPE_F64 = {256, 2, 1, 0, 0};
constexpr int N_STEP_SHAPES = 13;
// Staged shapes: threads per CTA (one producer warp, the rest consume), pipeline stages
// (tiles in flight per CTA), CTAs per SM and consumer groups (tiles worked on at once).
struct StagedShape { int threads, stages, ctas_per_sm, groups; };
constexpr StagedShape STAGED_SHAPES[2] = {{992, 3, 1, 2}, {512, 3, 1, 1}};
inline int staged_of(int variant) {
    return (variant >= 0 && variant < N_STEP_SHAPES) ? STEP_SHAPES[variant].staged - 1 : -1;
}
inline size_t esize_of_precision(int precision) {
    return precision == LBM_F64 ? 8 : (precision == LBM_F32 ? 4 : 2);
}
// Storage elements per direction segment of staged shape k: the largest multiple of 64
// whose STAGES stages (27 segments + a 16-byte cell-table entry per element each) and
// mbarriers fit the shared memory of one CTA when ctas_per_sm CTAs share an SM (GB300:
// 227 KB per CTA, 228 KB per SM with 1 KB reserved per CTA).
inline int staged_cap(int precision, int k) {
    const StagedShape &sh = STAGED_SHAPES[k];
    const int budget = (sh.ctas_per_sm == 1 ? 232448 : (233472 / sh.ctas_per_sm - 1024)) - 80 * sh.stages - 128;
    const int per = sh.stages * (27 * (int)esize_of_precision(precision) + 16);
    return budget / per / 64 * 64;
}
inline int step_variants(int) { return N_STEP_SHAPES; }
// the fastest shapes in sweeps on GB300: 128 x 8 threads with 2 planes per thread for
// F32 storage, with 4 planes for the 16-bit formats and for Bouzidi walls (with the link
// coefficients tabulated per wall link, 4 planes per thread beat one by 4 %)
inline int default_variant(int precision, int wall) {
    if (precision == LBM_F64) return 0;
    if (wall == LBM_BOUZIDI) return 7;
    return precision == LBM_F32 ? 6 : 7;
}
// the fastest shape of the odd (neighbour-slot) steps: 128 x 7 with 2 planes per thread
// (more registers for the 27 neighbour addresses and wall-link selects; R = 96 pipe: odd
// step 0.855 of measured HBM against 0.824 with the even steps' shape)
inline int default_variant_odd(int precision, int wall) {
    if (precision == LBM_F64) return 0;
    if (wall == LBM_BOUZIDI) return 7;
    return 9;
}
// the shape the ablation collision models are compiled for (one plane per thread)
inline int model_variant(int precision) { return precision == LBM_F64 ? 0 : 2; }
// the shape of the adjoint's moment-storing recompute (256 x 4, one plane per thread:
// two planes per thread measured 2 % slower there)
constexpr int MOM_VARIANT = 0;
inline int moments_variant(int) { return MOM_VARIANT; }
// whether the storage can run the shape at all (a staged shape also needs a compact pipe
// layout whose row groups fit its segments: checked per context)
inline bool step_variant_ok(int precision, int variant) {
    if (variant < 0 || variant >= N_STEP_SHAPES) return false;
    if (STEP_SHAPES[variant].staged) return true;
    if (precision == LBM_F64) return variant == 0;
    return precision == LBM_F32 || !STEP_SHAPES[variant].pipelined;
}
inline int step_threads(int precision, int variant) {
    if (precision == LBM_F64 && !STEP_SHAPES[variant].staged) return STEP_SHAPE_F64.threads;
    return STEP_SHAPES[variant].threads;
}
inline int step_zc(int precision, int variant) { return precision == LBM_F64 ? 1 : STEP_SHAPES[variant].zc; }

// Sets the shared-memory size of the staged step kernels of shape `variant` for every
// parity, wall and statistics setting of storage P (once per process; called before any
// graph capture so that the launches being captured only launch).
template <int P>
cudaError_t prepare_step(int wall, int variant);
// Step of a staged shape (lbm_staged.cuh; compiled in lbm_staged_*.cu).
template <int P>
cudaError_t launch_step_staged(int wall, int parity, bool stats, const StepArgs &a, int variant, cudaStream_t s);

// Every launcher enqueues on `s` and returns the launch status.
// Step kernel over all members: a flat grid of a.nblocks_total blocks of
// step_threads(P, variant) threads.
template <int P>
cudaError_t launch_step(int wall, int parity, bool stats, const StepArgs &a, int variant, cudaStream_t s);

// Forward step that also stores rho, u, s4..s8 into a.moments (adjoint recompute;
// single half-way pipe, F32 or F64 storage, in the shape moments_variant).
template <int P>
cudaError_t launch_step_moments(int parity, const StepArgs &a, cudaStream_t s);

// One backward step of the adjoint (see k_adjoint): 256-thread blocks, each thread
// takes ADJ_ZC consecutive planes of one stored position (two planes measured 7 %
// slower than one on GB300: the loop state spills at the kernel's register budget).
constexpr int ADJ_ZC = 1;
struct AdjArgs {
    const void *lam_next;     // lambda_{t+1}, [27][cells] in the compute type
    void *lam;                // lambda_t (written)
    const void *moments;      // [9][cells] of step t: rho, u_x, u_y, u_z, s4..s8
    double *acc;              // [cells]: dJ/dg_z (accumulated, FP64, dense cells)
    void *acc_seg;            // [stored cells]: dJ/dg_z of the current segment (compute type;
                              // added into acc and cleared after each segment)
    double *blockacc;         // [2][nblocks * 8]: objective and dJ/domega per warp (accumulated)
    int32_t objective;        // LBM_J_UBULK | LBM_J_WSS
    double kappa;             // UBULK: 1 / (T N_fluid)
    double wss;               // WSS: 2 / (T 2 pi R nz)
    float kappa_f, wss_f;     // the same in float
    int32_t nblocks;
};
template <int P>
cudaError_t launch_adjoint(const StepArgs &a, const AdjArgs &j, cudaStream_t s);
// acc[dense cell] += acc_seg[stored cell]; acc_seg = 0 (member 0 of a, compact layout).
template <int P>
cudaError_t launch_flush_segment(const StepArgs &a, const Member &hm, const AdjArgs &j, cudaStream_t s);
// Deterministic column sums of nv <= 5 double arrays [nv][n] into out[5] (device).
template <int P>
cudaError_t launch_sum_columns(const double *base, int64_t n, int nv, double *partials, int n_partials_max,
                               double *out, cudaStream_t s);

// Per-member kernels: member m of a.members (host copy hm for sizes).
template <int P>
cudaError_t launch_moments(int wall, int parity, const StepArgs &a, const Member &hm, int m,
                           void *rho, void *u, cudaStream_t s);
template <int P>
cudaError_t launch_get_pops(int wall, int parity, const StepArgs &a, const Member &hm, int m,
                            double *f, cudaStream_t s);
template <int P>
cudaError_t launch_set_pops(int wall, int parity, const StepArgs &a, const Member &hm, int m,
                            const double *f, cudaStream_t s);
template <int P>
cudaError_t launch_init(int wall, const StepArgs &a, const Member &hm, int m, int profile, double noise_amp,
                        uint64_t seed, const double *rho, const double *u, cudaStream_t s);
// Block partials (5 doubles per block) then a one-block final pass into out[5] (device).
template <int P>
cudaError_t launch_reduce(int wall, int parity, const StepArgs &a, const Member &hm, int m,
                          double *partials, int n_partials_max, double *out, cudaStream_t s);
template <int P>
cudaError_t launch_modes(int wall, int parity, const StepArgs &a, const Member &hm, int m,
                         const ModesArgs &ma, double *E, cudaStream_t s);

// Trigger-force tables of member m (column factors [3][ny][nx], z factors [2][nz]).
template <int P>
cudaError_t launch_force_tables(const Member *dmembers, const Member &hm, int m, void *ftab, void *ztab,
                                cudaStream_t s);

// Records the reason of a failed call that has no context (reported by
// lbm_last_error(NULL) in the calling thread).
void set_thread_error(const char *msg);

constexpr int REDUCE_BLOCK = 256;
constexpr int REDUCE_MAX_BLOCKS = 1216;   // 8 resident blocks x 152 SMs

}  // namespace lbm
