// lbm_kernels.cuh -- kernels of the pipe-flow LBM, instantiated once per storage
// precision by lbm_f64.cu, lbm_f32.cu, lbm_f16s.cu and lbm_bf16.cu (each defines
// LBM_PREC before including this file).
#pragma once

#include <algorithm>

#include "lbm_internal.h"

namespace lbm {

// ---- the fused step: load (stream) + wall + force + MRT collision + store ----------------
// One thread per cell of every member; solid cells return at once.  On sample
// steps (STATS) u_z^k, k = 1..4, of the pre-collision state is added in FP64.
// BS threads per block, register budget for MINB resident blocks per SM.
template <int P, int PAR, int WALL, bool STATS, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_step(const __grid_constant__ StepArgs a) {
    using R = typename Storage<P>::R;
    const int m = find_member(a, blockIdx.x);
    const Member &d = a.members[m];
    const uint32_t local = (uint32_t)(blockIdx.x - a.block0[m]) * BS + threadIdx.x;
    if (local >= (uint32_t)d.cells) return;
    CellPos p;
    cell_setup(d, local, p);
    if (!((p.nb >> 4) & 1u)) return;
    const int64_t t = a.times ? a.times[a.tidx].t : a.t;
    const double stv = a.times ? a.times[a.tidx].st[m] : a.st[m];
    R v[Q];
    load_pops<P, PAR, WALL>(a, d, p, v);
    R gx, gy, gz;
    acceleration<R>(d, p, t, stv, gx, gy, gz);
    const Macro<R> mm = collide<R>(v, gx, gy, gz, (R)d.omega);
    if constexpr (STATS) {
        const double uz = (double)mm.uz;
        double *s = a.stats + d.off + p.lc;
        const double uz2 = uz * uz;
        s[0] += uz;
        s[a.stride] += uz2;
        s[2 * a.stride] += uz2 * uz;
        s[3 * a.stride] += uz2 * uz2;
    }
    store_pops<P, PAR, WALL>(a, d, p, v);
}

// ---- state I/O: the exact inverse of load_pops ---------------------------------------------
template <int P, int PAR, int WALL>
__device__ __forceinline__ void write_state(const StepArgs &a, const Member &d, const CellPos &p,
                                            typename Storage<P>::R (&v)[Q]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    T *base = static_cast<T *>(a.pops);
    const R sc = (R)a.f16_scale;
    if constexpr (WALL == LBM_BOUZIDI) {
        if (p.nb != 0x1FFu) {
            sfor<0, Q>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if constexpr (cx_of(j) != 0 || cy_of(j) != 0) {
                    if (!dst_is_fluid<j>(p)) {
                        BLink<R> b = bouzidi_link<R, j>(d, p);
                        v[opp_of(j)] -= b.C * v[j];
                    }
                }
            });
        }
    }
    T *b = base + d.off;
    const uint32_t st = (uint32_t)a.stride;
    const uint32_t lc = (uint32_t)p.lc;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ib = opp_of(i);
        if constexpr (PAR == 0) {
            S::st(b + (i * st + lc), v[i], sc);
        } else {
            const uint32_t pull = ib * st + (uint32_t)(p.lc + src_offset<i>(p));
            if constexpr (WALL == LBM_FULLWAY || (cx_of(i) == 0 && cy_of(i) == 0)) {
                S::st(b + pull, v[i], sc);
            } else {
                const uint32_t own = i * st + lc;
                S::st(b + (src_is_fluid<i>(p) ? pull : own), v[i], sc);
            }
        }
    });
}

// Shifted equilibrium f^eq(rho, u) - w in the product form (no force term).
template <class R>
__device__ __forceinline__ void feq_shifted(R drho, R ux, R uy, R uz, R (&v)[Q]) {
    R dx[3], hx[3], dy[3], hy[3], dz[3], hz[3];
    axis_factors<R>(ux, R(0), dx, hx);
    axis_factors<R>(uy, R(0), dy, hy);
    axis_factors<R>(uz, R(0), dz, hz);
    const R rho = R(1) + drho;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const R dxy = dx[cx_of(i) + 1] + dy[cy_of(i) + 1] + dx[cx_of(i) + 1] * dy[cy_of(i) + 1];
        const R pm1 = dxy + dz[cz_of(i) + 1] * (R(1) + dxy);
        v[i] = R(w_of(i)) * (drho + rho * pm1);
    });
}

template <int P, int PAR, int WALL>
__global__ void k_moments(const __grid_constant__ StepArgs a, int m, typename Storage<P>::R *rho,
                          typename Storage<P>::R *u) {
    using R = typename Storage<P>::R;
    const Member &d = a.members[m];
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= d.cells) return;
    CellPos p;
    cell_setup(d, (uint32_t)local, p);
    if (!((p.nb >> 4) & 1u)) {
        rho[local] = 0;
        u[local] = 0;
        u[d.cells + local] = 0;
        u[2 * d.cells + local] = 0;
        return;
    }
    R v[Q];
    load_pops<P, PAR, WALL>(a, d, p, v);
    R gx, gy, gz;
    acceleration<R>(d, p, a.t, a.st[m], gx, gy, gz);
    const Macro<R> mm = macroscopic<R>(v, gx, gy, gz);
    rho[local] = mm.rho;
    u[local] = mm.ux;
    u[d.cells + local] = mm.uy;
    u[2 * d.cells + local] = mm.uz;
}

template <int P, int PAR, int WALL>
__global__ void k_get_pops(const __grid_constant__ StepArgs a, int m, double *f) {
    using R = typename Storage<P>::R;
    const Member &d = a.members[m];
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= d.cells) return;
    CellPos p;
    cell_setup(d, (uint32_t)local, p);
    R v[Q];
    if (((p.nb >> 4) & 1u) || WALL == LBM_FULLWAY) {
        load_pops<P, PAR, WALL>(a, d, p, v);
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = 0;
    }
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        f[(int64_t)i * d.cells + local] = (double)v[i] + w_of(i);
    });
}

template <int P, int PAR, int WALL>
__global__ void k_set_pops(const __grid_constant__ StepArgs a, int m, const double *f) {
    using R = typename Storage<P>::R;
    const Member &d = a.members[m];
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= d.cells) return;
    CellPos p;
    cell_setup(d, (uint32_t)local, p);
    if (!((p.nb >> 4) & 1u) && WALL != LBM_FULLWAY) return;
    R v[Q];
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        v[i] = (R)(f[(int64_t)i * d.cells + local] - w_of(i));
    });
    write_state<P, PAR, WALL>(a, d, p, v);
}

// ---- initial state ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea, Flood 2014): output n of seed s is mix64(s + (n+1) gamma).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t n) {
    uint64_t z = seed + (n + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Box-Muller normal number (3 c + k) for cell c, component k.
__device__ __forceinline__ double normal_at(uint64_t seed, uint64_t cell, int k) {
    const uint64_t n1 = 2ull * (3ull * cell + (uint64_t)k);
    const double u1 = ((double)(splitmix64_at(seed, n1) >> 11) + 1.0) * 0x1.0p-53;
    const double u2 = (double)(splitmix64_at(seed, n1 + 1ull) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

template <int P, int WALL>
__global__ void k_init(const __grid_constant__ StepArgs a, int m, int profile, double noise_amp,
                       uint64_t seed, const double *rho_in, const double *u_in) {
    using R = typename Storage<P>::R;
    const Member &d = a.members[m];
    const int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (local >= d.cells) return;
    CellPos p;
    cell_setup(d, (uint32_t)local, p);
    R v[Q];
    if (!((p.nb >> 4) & 1u)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = 0;
        write_state<P, 0, LBM_FULLWAY>(a, d, p, v);   // plain own-slot write at t = 0
        return;
    }
    double ux = 0, uy = 0, uz = 0, drho = 0;
    if (rho_in != nullptr) {
        drho = rho_in[local] - 1.0;
        ux = u_in[local];
        uy = u_in[d.cells + local];
        uz = u_in[2 * d.cells + local];
    } else {
        const double px = 0.5 * (double)(2 * p.x - d.nx + 1), py = 0.5 * (double)(2 * p.y - d.ny + 1);
        const double r = sqrt(px * px + py * py);
        const double nu = (1.0 / d.omega - 0.5) / 3.0;
        const double gz = d.g[2];
        if (profile == LBM_LAMINAR) {
            uz = gz * (d.R * d.R - r * r) / (4.0 * nu);
        } else if (profile == LBM_LOGLAW) {
            const double us = sqrt(gz * d.R / 2.0);
            const double dplus = (d.R - r) * us / nu;
            const double uplus = dplus <= 10.8 ? dplus : log(dplus) / 0.4 + 5.0;
            uz = us * uplus;
        }
        if (noise_amp != 0.0) {
            ux += noise_amp * normal_at(seed, (uint64_t)local, 0);
            uy += noise_amp * normal_at(seed, (uint64_t)local, 1);
            uz += noise_amp * normal_at(seed, (uint64_t)local, 2);
        }
    }
    feq_shifted<R>((R)drho, (R)ux, (R)uy, (R)uz, v);
    write_state<P, 0, WALL>(a, d, p, v);
}

// ---- reductions (deterministic two-pass) -------------------------------------------------------
template <int NV>
__device__ __forceinline__ void block_sum(double (&x)[NV], double *sh /* [NV][32] */) {
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_down_sync(0xFFFFFFFFu, x[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k * 32 + warp] = x[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            x[k] = lane < nw ? sh[k * 32 + lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x[k] += __shfl_down_sync(0xFFFFFFFFu, x[k], o);
        }
    }
}

template <int P, int PAR, int WALL>
__global__ void __launch_bounds__(REDUCE_BLOCK) k_reduce(const __grid_constant__ StepArgs a, int m,
                                                         double *partials) {
    using R = typename Storage<P>::R;
    __shared__ double sh[5 * 32];
    const Member &d = a.members[m];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t local = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; local < d.cells;
         local += (int64_t)gridDim.x * blockDim.x) {
        CellPos p;
        cell_setup(d, (uint32_t)local, p);
        if (!((p.nb >> 4) & 1u)) continue;
        R v[Q];
        load_pops<P, PAR, WALL>(a, d, p, v);
        double dr = 0, jx = 0, jy = 0, jz = 0;
        bool bad = false;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const double x = (double)v[i];
            bad |= !isfinite(x);
            dr += x;
            jx += cx_of(i) * x;
            jy += cy_of(i) * x;
            jz += cz_of(i) * x;
        });
        acc[0] += dr;
        acc[1] += jx;
        acc[2] += jy;
        acc[3] += jz;
        acc[4] += bad ? 1.0 : 0.0;
    }
    block_sum<5>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) partials[blockIdx.x * 5 + k] = acc[k];
}

static __global__ void __launch_bounds__(REDUCE_BLOCK) k_reduce_final(const double *partials, int n, double *out) {
    __shared__ double sh[5 * 32];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < n; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += partials[b * 5 + k];
    block_sum<5>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k] = acc[k];
}

// ---- coherent-structure rings, Sec. II.C -------------------------------------------------------
template <int P, int PAR, int WALL>
__device__ double uz_at(const StepArgs &a, const Member &d, int m, int x, int y, int z) {
    using R = typename Storage<P>::R;
    if (x < 0 || y < 0 || x >= d.nx || y >= d.ny) return 0.0;
    CellPos p;
    cell_setup(d, (uint32_t)(((int64_t)z * d.ny + y) * d.nx + x), p);
    if (!((p.nb >> 4) & 1u)) return 0.0;
    R v[Q];
    load_pops<P, PAR, WALL>(a, d, p, v);
    R gx, gy, gz;
    acceleration<R>(d, p, a.t, a.st[m], gx, gy, gz);
    return (double)macroscopic<R>(v, gx, gy, gz).uz;
}

// One block per (section, ring): bilinear samples of u_z into shared memory, then the
// DFT energies E_m = |sum_n u_n e^{-i m theta_n}|^2 / N^2 with warp-shuffle sums.
template <int P, int PAR, int WALL>
__global__ void k_modes(const __grid_constant__ StepArgs a, int m, const ModesArgs ma, double *E) {
    extern __shared__ double smp[];
    const Member &d = a.members[m];
    const int s = blockIdx.x / ma.n_rings, j = blockIdx.x % ma.n_rings;
    const int z = (int)(((int64_t)s * d.nz) / ma.n_sections);
    const int N = ma.n_theta;
    const double xc = 0.5 * (d.nx - 1), yc = 0.5 * (d.ny - 1);
    const double r = ma.r_over_R[j] * d.R;
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)n / (double)N, &sn, &cs);
        const double px = xc + r * cs, py = yc + r * sn;
        const int i0 = (int)floor(px), j0 = (int)floor(py);
        const double fx = px - i0, fy = py - j0;
        const double u00 = uz_at<P, PAR, WALL>(a, d, m, i0, j0, z);
        const double u10 = uz_at<P, PAR, WALL>(a, d, m, i0 + 1, j0, z);
        const double u01 = uz_at<P, PAR, WALL>(a, d, m, i0, j0 + 1, z);
        const double u11 = uz_at<P, PAR, WALL>(a, d, m, i0 + 1, j0 + 1, z);
        smp[n] = (1 - fx) * (1 - fy) * u00 + fx * (1 - fy) * u10 + (1 - fx) * fy * u01 + fx * fy * u11;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int mode = warp; mode <= ma.n_modes; mode += nw) {
        double re = 0, im = 0;
        for (int n = lane; n < N; n += 32) {
            const int64_t k = ((int64_t)mode * n) % N;
            double sn, cs;
            sincospi(2.0 * (double)k / (double)N, &sn, &cs);
            re += smp[n] * cs;
            im -= smp[n] * sn;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xFFFFFFFFu, re, o);
            im += __shfl_down_sync(0xFFFFFFFFu, im, o);
        }
        if (lane == 0)
            E[((int64_t)s * ma.n_rings + j) * (ma.n_modes + 1) + mode] = (re * re + im * im) / ((double)N * N);
    }
}

// ---- trigger-force tables ---------------------------------------------------------------------
template <class R>
__global__ void k_force_tables(const Member *members, int m, R *ftab, R *ztab) {
    const Member &d = members[m];
    const int ncol = d.nx * d.ny;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ncol) {
        double Px, Py, Pz;
        trigger_column(d, k % d.nx, k / d.nx, Px, Py, Pz);
        ftab[k] = (R)Px;
        ftab[ncol + k] = (R)Py;
        ftab[2 * ncol + k] = (R)Pz;
    }
    if (k < d.nz) {
        double sz, cz;
        sincospi(2.0 * (double)d.kz * (double)k / (double)d.nz, &sz, &cz);
        ztab[k] = (R)cz;
        ztab[d.nz + k] = (R)sz;
    }
}

// ---- host launchers ------------------------------------------------------------------------------
#define LBM_DISPATCH_WP(WALL_, PAR_, ...)                                          \
    do {                                                                          \
        if (WALL_ == LBM_HALFWAY) {                                               \
            if (PAR_ == 0) { constexpr int W = LBM_HALFWAY, PA = 0; __VA_ARGS__; } \
            else { constexpr int W = LBM_HALFWAY, PA = 1; __VA_ARGS__; }          \
        } else if (WALL_ == LBM_FULLWAY) {                                        \
            if (PAR_ == 0) { constexpr int W = LBM_FULLWAY, PA = 0; __VA_ARGS__; } \
            else { constexpr int W = LBM_FULLWAY, PA = 1; __VA_ARGS__; }          \
        } else {                                                                  \
            if (PAR_ == 0) { constexpr int W = LBM_BOUZIDI, PA = 0; __VA_ARGS__; } \
            else { constexpr int W = LBM_BOUZIDI, PA = 1; __VA_ARGS__; }          \
        }                                                                         \
    } while (0)

static inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <int P, int BS, int MINB>
cudaError_t launch_step_shape(int wall, int parity, bool stats, const StepArgs &a, cudaStream_t s) {
    LBM_DISPATCH_WP(wall, parity, {
        if (stats) k_step<P, PA, W, true, BS, MINB><<<a.nblocks_total, BS, 0, s>>>(a);
        else k_step<P, PA, W, false, BS, MINB><<<a.nblocks_total, BS, 0, s>>>(a);
    });
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_step(int wall, int parity, bool stats, const StepArgs &a, int variant, cudaStream_t s) {
    if (a.nblocks_total <= 0) return cudaSuccess;
    if constexpr (P == LBM_F64) {
        return launch_step_shape<P, 256, 2>(wall, parity, stats, a, s);
    } else {
        switch (variant) {
            case 1: return launch_step_shape<P, 256, 3>(wall, parity, stats, a, s);
            case 2: return launch_step_shape<P, 128, 8>(wall, parity, stats, a, s);
            case 3: return launch_step_shape<P, 512, 2>(wall, parity, stats, a, s);
            default: return launch_step_shape<P, 256, 4>(wall, parity, stats, a, s);
        }
    }
}

template <int P>
cudaError_t launch_moments(int wall, int parity, const StepArgs &a, const Member &hm, int m, void *rho,
                           void *u, cudaStream_t s) {
    using R = typename Storage<P>::R;
    if (hm.cells == 0) return cudaSuccess;
    LBM_DISPATCH_WP(wall, parity, {
        k_moments<P, PA, W><<<blocks_for(hm.cells, 256), 256, 0, s>>>(a, m, (R *)rho, (R *)u);
    });
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_get_pops(int wall, int parity, const StepArgs &a, const Member &hm, int m, double *f,
                            cudaStream_t s) {
    if (hm.cells == 0) return cudaSuccess;
    LBM_DISPATCH_WP(wall, parity, { k_get_pops<P, PA, W><<<blocks_for(hm.cells, 256), 256, 0, s>>>(a, m, f); });
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_set_pops(int wall, int parity, const StepArgs &a, const Member &hm, int m, const double *f,
                            cudaStream_t s) {
    if (hm.cells == 0) return cudaSuccess;
    LBM_DISPATCH_WP(wall, parity, { k_set_pops<P, PA, W><<<blocks_for(hm.cells, 256), 256, 0, s>>>(a, m, f); });
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_init(int wall, const StepArgs &a, const Member &hm, int m, int profile, double noise_amp,
                        uint64_t seed, const double *rho, const double *u, cudaStream_t s) {
    if (hm.cells == 0) return cudaSuccess;
    const unsigned nb = blocks_for(hm.cells, 256);
    if (wall == LBM_HALFWAY) k_init<P, LBM_HALFWAY><<<nb, 256, 0, s>>>(a, m, profile, noise_amp, seed, rho, u);
    else if (wall == LBM_FULLWAY) k_init<P, LBM_FULLWAY><<<nb, 256, 0, s>>>(a, m, profile, noise_amp, seed, rho, u);
    else k_init<P, LBM_BOUZIDI><<<nb, 256, 0, s>>>(a, m, profile, noise_amp, seed, rho, u);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_reduce(int wall, int parity, const StepArgs &a, const Member &hm, int m, double *partials,
                          int n_partials_max, double *out, cudaStream_t s) {
    int nb = (int)blocks_for(hm.cells, REDUCE_BLOCK);
    if (nb > n_partials_max) nb = n_partials_max;
    if (nb < 1) nb = 1;
    LBM_DISPATCH_WP(wall, parity, { k_reduce<P, PA, W><<<nb, REDUCE_BLOCK, 0, s>>>(a, m, partials); });
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, REDUCE_BLOCK, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_force_tables(const Member *dmembers, const Member &hm, int m, void *ftab, void *ztab,
                                cudaStream_t s) {
    using R = typename Storage<P>::R;
    const int n = (int)std::max<int64_t>((int64_t)hm.nx * hm.ny, hm.nz);
    k_force_tables<R><<<blocks_for(n, 256), 256, 0, s>>>(dmembers, m, (R *)ftab, (R *)ztab);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_modes(int wall, int parity, const StepArgs &a, const Member &hm, int m, const ModesArgs &ma,
                         double *E, cudaStream_t s) {
    (void)hm;
    const int nblk = ma.n_sections * ma.n_rings;
    const size_t shm = (size_t)ma.n_theta * sizeof(double);
    LBM_DISPATCH_WP(wall, parity, {
        if (shm > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_modes<P, PA, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e != cudaSuccess) return e;
        }
        k_modes<P, PA, W><<<nblk, 256, shm, s>>>(a, m, ma, E);
    });
    return cudaGetLastError();
}

}  // namespace lbm

// Explicit instantiation of every launcher for one storage precision.
#define LBM_INSTANTIATE(P)                                                                              \
    namespace lbm {                                                                                     \
    template cudaError_t launch_step<P>(int, int, bool, const StepArgs &, int, cudaStream_t);           \
    template cudaError_t launch_moments<P>(int, int, const StepArgs &, const Member &, int, void *,     \
                                           void *, cudaStream_t);                                       \
    template cudaError_t launch_get_pops<P>(int, int, const StepArgs &, const Member &, int, double *,  \
                                            cudaStream_t);                                              \
    template cudaError_t launch_set_pops<P>(int, int, const StepArgs &, const Member &, int,            \
                                            const double *, cudaStream_t);                              \
    template cudaError_t launch_init<P>(int, const StepArgs &, const Member &, int, int, double,        \
                                        uint64_t, const double *, const double *, cudaStream_t);        \
    template cudaError_t launch_reduce<P>(int, int, const StepArgs &, const Member &, int, double *,    \
                                          int, double *, cudaStream_t);                                 \
    template cudaError_t launch_modes<P>(int, int, const StepArgs &, const Member &, int,               \
                                         const ModesArgs &, double *, cudaStream_t);                    \
    template cudaError_t launch_force_tables<P>(const Member *, const Member &, int, void *, void *,     \
                                                cudaStream_t);                                          \
    }
