// lbm_analysis.cu -- statistics profiles, dominant modes and the stochastic analysis of
// the dominant-mode series (Sec. III.B and Sec. III.C).
#include <cmath>
#include <cstring>
#include <vector>

#include "lbm.h"
#include "lbm_device.cuh"

namespace {

// Per-cell central moments from the raw sums S_k = sum u_z^k over `count` samples:
// mean, rms = <du^2>^(1/2), S3 = <du^3> / rms^3, S4 = <du^4> / rms^4 (du = u - <u>_t),
// accumulated per radial bin (bin = floor(r / dr)): [nbins][5] = count, sum of mean,
// rms, S3, S4.
__global__ void k_stats_profile(const double *acc, int64_t stride, int nx, int ny, int nz, double count,
                                const uint16_t *colmask, int nbins, double dr, double *bins) {
    extern __shared__ double sb[];
    for (int k = threadIdx.x; k < nbins * 5; k += blockDim.x) sb[k] = 0.0;
    __syncthreads();
    const int64_t cells = (int64_t)nx * ny * nz;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % nx), y = (int)((c / nx) % ny);
        if (!((colmask[y * nx + x] >> 4) & 1u)) continue;
        const double px = 0.5 * (2 * x - nx + 1), py = 0.5 * (2 * y - ny + 1);
        const int b = (int)(sqrt(px * px + py * py) / dr);
        if (b >= nbins) continue;
        const double s1 = acc[c] / count, s2 = acc[stride + c] / count;
        const double s3 = acc[2 * stride + c] / count, s4 = acc[3 * stride + c] / count;
        const double mu = s1;
        const double var = s2 - mu * mu;
        const double m3 = s3 - 3.0 * mu * s2 + 2.0 * mu * mu * mu;
        const double m4 = s4 - 4.0 * mu * s3 + 6.0 * mu * mu * s2 - 3.0 * mu * mu * mu * mu;
        const double rms = sqrt(var > 0.0 ? var : 0.0);
        const double S3 = rms > 0.0 ? m3 / (rms * rms * rms) : 0.0;
        const double S4 = rms > 0.0 ? m4 / (rms * rms * rms * rms) : 0.0;
        atomicAdd(&sb[b * 5 + 0], 1.0);
        atomicAdd(&sb[b * 5 + 1], mu);
        atomicAdd(&sb[b * 5 + 2], rms);
        atomicAdd(&sb[b * 5 + 3], S3);
        atomicAdd(&sb[b * 5 + 4], S4);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nbins * 5; k += blockDim.x)
        if (sb[k] != 0.0) atomicAdd(&bins[k], sb[k]);
}

}  // namespace

// Internal entry used by lbm_api.cu (keeps the kernel in this file).
cudaError_t lbm_launch_stats_profile(const double *acc, int64_t stride, const lbm::Member &d, double count, int nbins,
                                     double dr, double *bins, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(double) * 5 * nbins, s);
    if (e != cudaSuccess) return e;
    k_stats_profile<<<304, 256, sizeof(double) * 5 * nbins, s>>>(acc, stride, d.nx, d.ny, d.nz, count, d.colmask,
                                                                  nbins, dr, bins);
    return cudaGetLastError();
}

extern "C" {

int lbm_dominant_modes(const double *E, int32_t n_sections, int32_t n_rings, int32_t n_modes, int32_t ring,
                       int32_t m_lo, int32_t m_hi, int32_t *kstar) {
    if (!E || !kstar || n_sections < 1 || n_rings < 1 || ring < 0 || ring >= n_rings || m_lo < 0 ||
        m_hi < m_lo || m_hi > n_modes)
        return LBM_EINVAL;
    for (int s = 0; s < n_sections; ++s) {
        const double *e = E + ((int64_t)s * n_rings + ring) * (n_modes + 1);
        int best = m_lo;
        for (int m = m_lo + 1; m <= m_hi; ++m)
            if (e[m] > e[best]) best = m;       // ties keep the smallest mode
        kstar[s] = best;
    }
    return LBM_OK;
}

int lbm_transition_matrix(const int32_t *series, int64_t n, int32_t m_lo, int32_t m_hi, int32_t lag, double *T,
                          int64_t *counts) {
    if (!series || !T || n < 0 || m_hi < m_lo || lag < 1) return LBM_EINVAL;
    const int K = m_hi - m_lo + 1;
    std::vector<int64_t> c((size_t)K * K, 0);
    for (int64_t t = 0; t + lag < n; ++t) {
        const int a = series[t], b = series[t + lag];
        if (a < m_lo || a > m_hi || b < m_lo || b > m_hi) continue;
        c[(size_t)(b - m_lo) * K + (a - m_lo)] += 1;      // row: destination i, column: origin j
    }
    for (int j = 0; j < K; ++j) {
        int64_t col = 0;
        for (int i = 0; i < K; ++i) col += c[(size_t)i * K + j];
        for (int i = 0; i < K; ++i) T[(size_t)i * K + j] = col > 0 ? (double)c[(size_t)i * K + j] / (double)col : 0.0;
    }
    if (counts) std::memcpy(counts, c.data(), sizeof(int64_t) * c.size());
    return LBM_OK;
}

int lbm_mode_correlation(const int32_t *series, int64_t n, int32_t m_lo, int32_t m_hi, int32_t max_lag, double *F) {
    if (!series || !F || n < 1 || m_hi < m_lo || max_lag < 0 || max_lag >= n) return LBM_EINVAL;
    const int K = m_hi - m_lo + 1;
    for (int k = 0; k < K; ++k) {
        const int m = m_lo + k;
        int64_t hits = 0;
        for (int64_t t = 0; t < n; ++t) hits += series[t] == m;
        const double p = (double)hits / (double)n;
        for (int lag = 0; lag <= max_lag; ++lag) {
            int64_t both = 0;
            for (int64_t t = 0; t + lag < n; ++t) both += (series[t] == m) && (series[t + lag] == m);
            F[(size_t)k * (max_lag + 1) + lag] = (double)both / (double)(n - lag) - p * p;
        }
    }
    return LBM_OK;
}

}  // extern "C"
