// lbm_static.cu -- lbm_reduce_static: the mass/momentum reduction without any allocation.
//
// Some callers cannot allocate device memory when they need this sum: an application
// whose device memory is owned entirely by its own pool (sized once at start-up, no
// outside cudaMalloc allowed), or a latency-critical loop that must not pay for the
// device-wide synchronisation a cudaMalloc/cudaFree implies.  For them the block
// partials of the two-pass reduction live in the fixed array below, which is part of
// the library image: every GPU that loads the library holds it until the process exits.
//
// The array is shared by every call on a device and keeps the last call's contents.
// Each call overwrites exactly the partials it then reads, so nothing has to start at
// zero.  Calls whose kernels overlap on the GPU (two streams, or two host threads on
// one device) race on the array: callers must order them, e.g. on one stream.
#include <cmath>
#include <mutex>

#include "lbm.h"
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace {

constexpr int SR_BLOCK = 256;

// Block partials (5 doubles per block) followed by the 5 final sums.
static __device__ __align__(256) double g_static_scratch[LBM_STATIC_REDUCE_MAX_BLOCKS * 5 + 8];

template <int P>
__global__ void __launch_bounds__(SR_BLOCK) k_reduce_static(const void *pops, uint32_t n, float inv,
                                                            double *scratch) {
    using S = lbm::Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    __shared__ double sh[5 * 32];
    const T *f = static_cast<const T *>(pops);
    double acc[5] = {0, 0, 0, 0, 0};
    for (uint32_t c = blockIdx.x * SR_BLOCK + threadIdx.x; c < n; c += gridDim.x * SR_BLOCK) {
        double dr = 0, jx = 0, jy = 0, jz = 0;
        bool bad = false;
        lbm::sfor<0, lbm::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const double x = (double)S::ld(f + (uint32_t)i * n + c, (R)inv);
            bad |= !isfinite(x);
            dr += x;
            jx += lbm::cx_of(i) * x;
            jy += lbm::cy_of(i) * x;
            jz += lbm::cz_of(i) * x;
        });
        acc[0] += dr;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        acc[4] += bad ? 1.0 : 0.0;
    }
    // warp, then block sums in a fixed order
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xFFFFFFFFu, acc[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) sh[k * 32 + warp] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double x = lane < SR_BLOCK / 32 ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
            if (lane == 0) scratch[blockIdx.x * 5 + k] = x;
        }
    }
}

__global__ void __launch_bounds__(SR_BLOCK) k_reduce_static_final(const double *scratch, int nblocks,
                                                                  double *out) {
    __shared__ double sh[5 * 32];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += SR_BLOCK)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += scratch[b * 5 + k];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xFFFFFFFFu, acc[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) sh[k * 32 + warp] = acc[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double x = lane < SR_BLOCK / 32 ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xFFFFFFFFu, x, o);
            if (lane == 0) out[k] = x;
        }
    }
}

// Device address of g_static_scratch, looked up once per device (with that device
// current) and cached.  In host code the array's name is only a host-side stand-in.
constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double *g_addr[MAX_DEVICES] = {};

int fail(int code, const char *why) {
    lbm::set_thread_error(why);
    return code;
}

// Device or managed memory (a host array handed to the kernel would fault or, where the
// GPU can reach host memory, be read through the wrong path).
bool device_reachable(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int lbm_reduce_static(const void *pops, int32_t precision, int32_t f16_log2_scale, int64_t n_cells,
                                 double *out, void *stream) {
    if (!pops || !out) return fail(LBM_EINVAL, "pops and out must not be NULL");
    if (n_cells < 1) return fail(LBM_EINVAL, "n_cells must be >= 1");
    if (n_cells > LBM_STATIC_REDUCE_MAX_CELLS)
        return fail(LBM_EINVAL, "n_cells exceeds LBM_STATIC_REDUCE_MAX_CELLS (27 x n_cells must stay below 2^32)");
    if (precision < LBM_F64 || precision > LBM_BF16) return fail(LBM_EINVAL, "unknown precision");
    int s16 = f16_log2_scale == 0 ? 16 : f16_log2_scale;
    if (s16 < 1 || s16 > 24) return fail(LBM_EINVAL, "f16_log2_scale must be in 1..24");
    if (!device_reachable(pops)) return fail(LBM_EINVAL, "pops must be device (or managed) memory");
    if (!device_reachable(out)) return fail(LBM_EINVAL, "out must be device (or managed) memory (5 doubles)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return fail(LBM_ECUDA, "no usable current CUDA device");
    }
    double *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(LBM_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
            }
            g_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_addr[dev];
    }
    const uint32_t n = (uint32_t)n_cells;
    int nb = (int)((n_cells + SR_BLOCK - 1) / SR_BLOCK);
    if (nb > LBM_STATIC_REDUCE_MAX_BLOCKS) nb = LBM_STATIC_REDUCE_MAX_BLOCKS;
    const float inv = std::ldexp(1.0f, -s16);
    cudaStream_t s = (cudaStream_t)stream;
    switch (precision) {
        case LBM_F64: k_reduce_static<LBM_F64><<<nb, SR_BLOCK, 0, s>>>(pops, n, inv, scratch); break;
        case LBM_F32: k_reduce_static<LBM_F32><<<nb, SR_BLOCK, 0, s>>>(pops, n, inv, scratch); break;
        case LBM_F16S: k_reduce_static<LBM_F16S><<<nb, SR_BLOCK, 0, s>>>(pops, n, inv, scratch); break;
        default: k_reduce_static<LBM_BF16><<<nb, SR_BLOCK, 0, s>>>(pops, n, inv, scratch); break;
    }
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA, "reduction kernel launch failed");
    k_reduce_static_final<<<1, SR_BLOCK, 0, s>>>(scratch, nb, out);
    if (cudaGetLastError() != cudaSuccess) return fail(LBM_ECUDA, "final reduction launch failed");
    return LBM_OK;
}
