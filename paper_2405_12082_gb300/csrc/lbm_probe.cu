// lbm_probe.cu -- lbm_probe_fp32: the measured FP32 arithmetic rate of the device.
//
// The step's roofline has two candidate bounds: DRAM bandwidth (the measured copy rate)
// and instruction issue (its FP32 collision, address arithmetic, loads and stores).  The
// copy rate is measured elsewhere; this probe measures the other side on the same GPU:
// kernels of independent fused multiply-adds that fill every SM (8 blocks of 256 threads
// each, 8 chains per thread, the loops unrolled 16 times), in scalar form (FFMA) and in
// Blackwell's paired form (two FMAs per instruction, __ffma2_rn), timed with CUDA events.  The chains never feed a store except under a
// condition the host makes false (a NaN sentinel), so nothing is optimised away and the
// kernels write no memory.
#include <cmath>

#include "lbm.h"
#include "lbm_internal.h"

namespace {

constexpr int PROBE_BLOCK = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;     // 2048 threads: a full SM
constexpr int PROBE_CHAINS = 8;            // independent dependency chains per thread

static __device__ float g_probe_sink;

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_ffma(float a, float b, int iters, float sentinel) {
    float x[PROBE_CHAINS];
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k];
    if (s == sentinel) g_probe_sink = s;
}

__global__ void __launch_bounds__(PROBE_BLOCK) k_probe_ffma2(float a, float b, int iters, float sentinel) {
    float2 x[PROBE_CHAINS];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k)
        x[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)(threadIdx.x + 2 * k) * 1e-3f);
#pragma unroll 16
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < PROBE_CHAINS; ++k) x[k] = __ffma2_rn(x[k], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) s += x[k].x + x[k].y;
    if (s == sentinel) g_probe_sink = s;
}

int fail(int code, const char *why) {
    lbm::set_thread_error(why);
    return code;
}

}  // namespace

extern "C" int lbm_probe_fp32(double *out, void *stream) {
    if (!out) return fail(LBM_EINVAL, "out must not be NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms < 1) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "no CUDA device");
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return fail(LBM_ECUDA, "cannot create CUDA events");
    }
    const int blocks = sms * PROBE_BLOCKS_PER_SM;
    const double threads = (double)blocks * PROBE_BLOCK;
    const float a = 0.99990f, b = 1.0e-3f, sentinel = std::nanf("");
    // the best of three timed launches after one untimed launch; returns ms or < 0 on error
    auto best_ms = [&](bool paired, int iters) -> float {
        float best = -1.0f;
        for (int r = 0; r < 4; ++r) {
            if (cudaEventRecord(e0, s) != cudaSuccess) return -1.0f;
            if (paired) k_probe_ffma2<<<blocks, PROBE_BLOCK, 0, s>>>(a, b, iters, sentinel);
            else k_probe_ffma<<<blocks, PROBE_BLOCK, 0, s>>>(a, b, iters, sentinel);
            if (cudaGetLastError() != cudaSuccess || cudaEventRecord(e1, s) != cudaSuccess ||
                cudaEventSynchronize(e1) != cudaSuccess)
                return -1.0f;
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0f;
            if (r > 0 && (best < 0.0f || ms < best)) best = ms;
        }
        return best;
    };
    const int iters1 = 1 << 18, iters2 = 1 << 17;
    const float ms1 = best_ms(false, iters1);
    const float ms2 = ms1 > 0.0f ? best_ms(true, iters2) : -1.0f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms1 <= 0.0f || ms2 <= 0.0f) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "the FP32 probe kernels failed to run");
    }
    const double fma1 = threads * iters1 * PROBE_CHAINS;          // scalar FMAs (one per instruction)
    const double fma2 = threads * iters2 * PROBE_CHAINS * 2.0;    // paired: two per instruction
    out[0] = 2.0 * fma1 / (ms1 * 1e-3) / 1e12;
    out[1] = 2.0 * fma2 / (ms2 * 1e-3) / 1e12;
    out[2] = fma1 / 32.0 / (ms1 * 1e-3) / (4.0 * sms);            // warp FFMA per second per sub-partition
    out[3] = ms1;
    return LBM_OK;
}
