// lbm_kernels.cuh -- kernels of the pipe-flow LBM, instantiated once per storage
// precision by lbm_f64.cu, lbm_f32.cu, lbm_f16s.cu and lbm_bf16.cu (each defines
// LBM_PREC before including this file).
#pragma once

#include <algorithm>
#include <type_traits>

#include "lbm_internal.h"

namespace lbm {

// ---- the fused step: load (stream) + wall + force + MRT collision + store ----------------
// One thread per cell of every member; solid cells return at once.  EXTRA selects
// what else the step does: EX_STATS adds u_z^k, k = 1..4, of the pre-collision state to
// the FP64 sums (sample steps); EX_MOMENTS stores rho, u and s4..s8 of the
// pre-collision state for the adjoint sweep.  BS threads per block, register budget
// for MINB resident blocks per SM.
enum { EX_NONE = 0, EX_STATS = 1, EX_MOMENTS = 2 };
#ifndef LBM_ADJ_MIN_BLOCKS
#define LBM_ADJ_MIN_BLOCKS 3
#endif

// Whether the step's populations travel in storage units (the scaled half format with the
// default collision: the scale is applied inside collide, see there).
template <int P, int EXTRA, int MODEL>
__host__ __device__ constexpr bool raw_units() {
    return Storage<P>::kScaled && MODEL == MODEL_MRT_H6 && EXTRA != EX_MOMENTS;
}

// Force, collide and store one fluid cell p of member d whose 27 populations (f - w, or
// (f - w) 2^s in raw units) are in v.
template <int P, int PAR, int WALL, int EXTRA, int MODEL>
__device__ __forceinline__ void finish_cell(const StepArgs &a, const Member &d, const CellPos &p, int64_t t,
                                            typename Storage<P>::R stv, typename Storage<P>::R (&v)[Q]) {
    using R = typename Storage<P>::R;
    R gx, gy, gz;
    acceleration<R>(d, p, t, stv, gx, gy, gz);
    if constexpr (EXTRA == EX_MOMENTS) {
        R sk[5];
        const Macro<R> mm = collide<R>(v, gx, gy, gz, omega_of<R>(d), sk);
        R *mo = static_cast<R *>(a.moments) + p.lc;
        const int64_t n = d.scells;
        mo[0] = mm.rho;
        mo[n] = mm.ux;
        mo[2 * n] = mm.uy;
        mo[3 * n] = mm.uz;
#pragma unroll
        for (int k = 0; k < 5; ++k) mo[(4 + k) * n] = sk[k];
    } else {
        constexpr bool SC = Storage<P>::kScaled && MODEL == MODEL_MRT_H6;
        const Macro<R> mm = collide<R, MODEL, SC>(v, gx, gy, gz, omega_of<R>(d), nullptr, lam1_of<R>(d),
                                                  (R)a.f16_inv, (R)a.f16_scale);
        if constexpr (EXTRA == EX_STATS) {
            const double uz = (double)mm.uz;
            double *s = a.stats + d.doff + p.di;
            const double uz2 = uz * uz;
            s[0] += uz;
            s[a.dstride] += uz2;
            s[2 * a.dstride] += uz2 * uz;
            s[3 * a.dstride] += uz2 * uz2;
        }
    }
    store_pops<P, PAR, WALL, raw_units<P, EXTRA, MODEL>()>(a, d, p, v);
}

// Stream, force, collide and store one fluid cell p of member d.
template <int P, int PAR, int WALL, int EXTRA, int MODEL>
__device__ __forceinline__ void step_cell(const StepArgs &a, const Member &d, const CellPos &p, int64_t t,
                                          typename Storage<P>::R stv) {
    using R = typename Storage<P>::R;
    R v[Q];
    load_pops<P, PAR, WALL, raw_units<P, EXTRA, MODEL>()>(a, d, p, v);
    finish_cell<P, PAR, WALL, EXTRA, MODEL>(a, d, p, t, stv, v);
}

// The cell above p (z + 1) in the same column: same in-plane data, one plane further.
__device__ __forceinline__ void next_plane(const Member &d, CellPos &p) {
    p.z += 1;
    p.lc += d.Ps;
    p.di += d.nx * d.ny;
    p.oz[0] = p.z == 0 ? (d.nz - 1) * d.Ps : -d.Ps;
    p.oz[2] = p.z == d.nz - 1 ? -(d.nz - 1) * d.Ps : d.Ps;
}

// ZC > 1: each thread takes ZC consecutive planes of one in-plane position (threads of a
// block stay consecutive in that position, so accesses stay coalesced); the position's
// table lookup and neighbour offsets are paid once per ZC cells.
template <int P, int PAR, int WALL, int EXTRA, int BS, int MINB, int MODEL = MODEL_MRT_H6, int ZC = 1>
__global__ void __launch_bounds__(BS, MINB) k_step(const __grid_constant__ StepArgs a) {
    using R = typename Storage<P>::R;
    const int m = find_member(a, blockIdx.x);
    const Member &d = a.members[m];
    const uint32_t local = (uint32_t)(blockIdx.x - a.block0[m]) * BS + threadIdx.x;
    if constexpr (ZC == 1) {
        if (local >= (uint32_t)d.scells) return;
        CellPos p;
        if (!cell_from_storage(d, local, p)) return;
        const int64_t t = a.times ? a.times[a.tidx].t : a.t;
        step_cell<P, PAR, WALL, EXTRA, MODEL>(a, d, p, t, st_of<R>(a, m));
    } else {
        const uint32_t nzg = (uint32_t)(d.nz + ZC - 1) / ZC;
        if (local >= (uint32_t)d.Ps * nzg) return;
        const uint32_t zg = fastdiv(local, d.ps_mul, d.ps_shr);
        const uint32_t r = local - zg * (uint32_t)d.Ps;
        CellPos p;
        if (!cell_from_storage(d, zg * ZC * (uint32_t)d.Ps + r, p)) return;
        const int64_t t = a.times ? a.times[a.tidx].t : a.t;
        const R stv = st_of<R>(a, m);
#pragma unroll 1
        for (int k = 0; k < ZC; ++k) {
            if (k > 0) {
                if (p.z + 1 >= d.nz) break;
                next_plane(d, p);
            }
            step_cell<P, PAR, WALL, EXTRA, MODEL>(a, d, p, t, stv);
        }
    }
}

// ---- software-pipelined persistent step (F32, F64 storage) -----------------------------------
// A persistent block walks over tiles of BS cells (grid-stride).  Before computing tile k
// each thread issues the 27 loads of its cell in tile k + 1 as cp.async copies into its
// own shared-memory column (stage (k+1) mod 2), so the loads of the next tile are in
// flight while the current one is computed, without holding registers.  Every AA slot is
// read and written by one cell only within a step, so prefetching ahead of other cells'
// stores is safe, and each thread reads back only what it copied itself: per-thread
// cp.async groups replace any block barrier.
__device__ __forceinline__ void cp_async_4(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

extern __shared__ __align__(16) unsigned char lbm_smem[];

template <int P, int PAR, int WALL>
__device__ __forceinline__ void prefetch_pops(const StepArgs &a, const Member &d, const CellPos &p, uint32_t sbase,
                                              int stride_bytes) {
    using T = typename Storage<P>::T;
    const T *base = static_cast<const T *>(a.pops) + d.off;
    const uint32_t st = (uint32_t)a.stride;
    const uint32_t lc = (uint32_t)p.lc;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ib = opp_of(i);
        uint32_t idx;
        if constexpr (PAR == 0) {
            idx = i * st + lc;
        } else {
            const uint32_t pull = ib * st + (uint32_t)(p.lc + src_offset<i>(p));
            if constexpr (WALL == LBM_FULLWAY || (cx_of(i) == 0 && cy_of(i) == 0)) idx = pull;
            else idx = src_is_fluid<i>(p) ? pull : i * st + lc;
        }
        if constexpr (sizeof(T) == 8) cp_async_8(sbase + i * stride_bytes, base + idx);
        else cp_async_4(sbase + i * stride_bytes, base + idx);
    });
}

struct TileCell {
    int m;
    bool active;
    CellPos p;
};

template <int BS>
__device__ __forceinline__ TileCell tile_cell(const StepArgs &a, int tile) {
    TileCell c;
    c.m = 0;
    c.active = false;
    if (tile < a.nblocks_total) {
        c.m = find_member(a, tile);
        const Member &d = a.members[c.m];
        const uint32_t local = (uint32_t)(tile - a.block0[c.m]) * BS + threadIdx.x;
        if (local < (uint32_t)d.scells) c.active = cell_from_storage(d, local, c.p);
    }
    return c;
}

template <int P, int PAR, int WALL, int EXTRA, int BS, int MINB>
__global__ void __launch_bounds__(BS, MINB) k_step_pipe(const __grid_constant__ StepArgs a) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const uint32_t smem0 = (uint32_t)__cvta_generic_to_shared(lbm_smem);
    const int stride_bytes = BS * (int)sizeof(T);            // one population column of a stage
    const uint32_t stage_bytes = (uint32_t)(Q * BS * sizeof(T));
    const uint32_t mine = smem0 + threadIdx.x * sizeof(T);
    const T *smem_t = reinterpret_cast<const T *>(lbm_smem) + threadIdx.x;
    int tile = blockIdx.x;
    TileCell cur = tile_cell<BS>(a, tile);
    if (cur.active) prefetch_pops<P, PAR, WALL>(a, a.members[cur.m], cur.p, mine, stride_bytes);
    cp_async_commit();
    const int64_t t = a.times ? a.times[a.tidx].t : a.t;
    for (int k = 0; tile < a.nblocks_total; ++k) {
        const int next_tile = tile + gridDim.x;
        TileCell nxt = tile_cell<BS>(a, next_tile);
        if (nxt.active)
            prefetch_pops<P, PAR, WALL>(a, a.members[nxt.m], nxt.p, mine + ((k + 1) & 1) * stage_bytes, stride_bytes);
        cp_async_commit();
        cp_async_wait_one();                                 // this thread's copies of tile k are done
        if (cur.active) {
            const Member &d = a.members[cur.m];
            const T *col = smem_t + (k & 1) * (Q * BS);
            R v[Q];
            const R inv = (R)a.f16_inv;
            sfor<0, Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                v[i] = S::ld(col + i * BS, inv);
            });
            if constexpr (WALL == LBM_BOUZIDI) bouzidi_load_fix<R>(d, cur.p, v);
            R gx, gy, gz;
            acceleration<R>(d, cur.p, t, st_of<R>(a, cur.m), gx, gy, gz);
            const Macro<R> mm = collide<R>(v, gx, gy, gz, omega_of<R>(d));
            if constexpr (EXTRA == EX_STATS) {
                const double uz = (double)mm.uz;
                double *sp = a.stats + d.doff + cur.p.di;
                const double uz2 = uz * uz;
                sp[0] += uz;
                sp[a.dstride] += uz2;
                sp[2 * a.dstride] += uz2 * uz;
                sp[3 * a.dstride] += uz2 * uz2;
            }
            store_pops<P, PAR, WALL>(a, d, cur.p, v);
        }
        tile = next_tile;
        cur = nxt;
    }
    cp_async_wait_all();
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

// Shifted second-order equilibrium f^eq(rho, u) - w (no force term).
template <class R>
__device__ __forceinline__ void feq_shifted_o2(R drho, R ux, R uy, R uz, R (&v)[Q]) {
    const R rho = R(1) + drho, uu = ux * ux + uy * uy + uz * uz;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const R cu = cterm<cz_of(i)>(cterm<cy_of(i)>(cterm<cx_of(i)>(R(-0.0), ux), uy), uz);
        v[i] = R(w_of(i)) * (drho + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu));
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
    if (!cell_from_dense(d, (uint32_t)local, p)) {
        rho[local] = 0;
        u[local] = 0;
        u[d.cells + local] = 0;
        u[2 * d.cells + local] = 0;
        return;
    }
    R v[Q];
    load_pops<P, PAR, WALL>(a, d, p, v);
    R gx, gy, gz;
    acceleration<R>(d, p, a.t, st_of<R>(a, m), gx, gy, gz);
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
    const bool fluid = cell_from_dense(d, (uint32_t)local, p);
    R v[Q];
    if (fluid || WALL == LBM_FULLWAY) {
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
    if (!cell_from_dense(d, (uint32_t)local, p) && WALL != LBM_FULLWAY) return;
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
    R v[Q];
    if (!cell_from_dense(d, (uint32_t)local, p)) {
        if (!d.compact) {                               // solid cells are stored only densely
#pragma unroll
            for (int i = 0; i < Q; ++i) v[i] = 0;
            write_state<P, 0, LBM_FULLWAY>(a, d, p, v);   // plain own-slot write at t = 0
        }
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
    if (a.collision & MODEL_O2) feq_shifted_o2<R>((R)drho, (R)ux, (R)uy, (R)uz, v);
    else feq_shifted<R>((R)drho, (R)ux, (R)uy, (R)uz, v);
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
        if (!cell_from_dense(d, (uint32_t)local, p)) continue;
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
    if (!cell_from_dense(d, (uint32_t)(((int64_t)z * d.ny + y) * d.nx + x), p)) return 0.0;
    R v[Q];
    load_pops<P, PAR, WALL>(a, d, p, v);
    R gx, gy, gz;
    acceleration<R>(d, p, a.t, st_of<R>(a, m), gx, gy, gz);
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

// ---- adjoint step ------------------------------------------------------------------------------
// Reverse of step t of a single half-way pipe.  mu = S^T lambda_{t+1} gathers
// lambda_i(x + c_i) when x + c_i is fluid and lambda_ibar(x) across a wall link (the
// transpose of half-way bounce-back); the wall-shear objective adds 2 c_iz / (T A_w) on
// wall links.  The collision is a function of rho, u and the raw shear moments m4..m8:
//   f*_j = w_j (rho P_j - 1) + (rho / 2) w_j g . grad_u P_j + (1 - omega) sum_k C_kj s_k,
//   P_j = psi(c_jx, u_x) psi(c_jy, u_y) psi(c_jz, u_z) (normalised), s_k = m_k - rho e_k(u)
//   + rho r_k(u, g) / 2,
// so lambda_t,i = A_rho + sum_a A_ua (c_ia - v_a) / rho + (1 - omega) sum_k q_k M_k(c_i)
// with v = u - g / 2, q_k = sum_j mu_j C_kj and A_rho, A_u the partial derivatives of
// sum_j mu_j f*_j.  The sums over j of mu_j w_j times products of psi and its first two
// u-derivatives are contracted axis by axis (z, then y, then x).  Per cell the FP64
// accumulators collect the objective, dJ/dg_z(x) and dJ/domega.
template <int P, int OBJ>
__device__ __forceinline__ void adjoint_cell(const StepArgs &a, const AdjArgs &j, const Member &d, const CellPos &p,
                                             typename Storage<P>::R &jterm, typename Storage<P>::R &wterm) {
    using R = typename Storage<P>::R;
    const uint32_t n = (uint32_t)d.scells, lc = (uint32_t)p.lc;
    const R *M = static_cast<const R *>(j.moments) + lc;
    const R rho = M[0], ux = M[n], uy = M[2 * n], uz = M[3 * n];
    const R s4 = M[4 * n], s5 = M[5 * n], s6 = M[6 * n], s7 = M[7 * n], s8 = M[8 * n];
    R gx, gy, gz;
    acceleration<R>(d, p, a.t, st_of<R>(a, 0), gx, gy, gz);
    const R om1 = R(1) - omega_of<R>(d);
    const R half = R(0.5);

    // mu = S^T lambda_{t+1} (+ wall shear source)
    const R wss = sizeof(R) == 4 ? (R)j.wss_f : (R)j.wss;
    const R *ln = static_cast<const R *>(j.lam_next);
    R mu[Q];
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ib = opp_of(i);
        const uint32_t push = i * n + (uint32_t)(p.lc + nb_offset<i>(p));
        if constexpr (cx_of(i) == 0 && cy_of(i) == 0) {
            mu[i] = ln[push];
        } else {
            const bool f = dst_is_fluid<i>(p);
            mu[i] = ln[f ? push : ib * n + lc];
            if constexpr (OBJ == LBM_J_WSS && cz_of(i) != 0)
                if (!f) mu[i] += wss * R(cz_of(i));
        }
    });

    // axis factors psi, psi', psi'' at c = -1, 0, +1
    R X0[3], X1[3], Y0[3], Y1[3], Z0[3], Z1[3];
    auto fac = [&](R u, R (&F0)[3], R (&F1)[3]) {
        const R u2 = u * u;
        F0[1] = R(1) - R(1.5) * u2;
        F0[0] = R(1) - R(3) * u + R(3) * u2;
        F0[2] = R(1) + R(3) * u + R(3) * u2;
        F1[1] = R(-3) * u;
        F1[0] = R(-3) + R(6) * u;
        F1[2] = R(3) + R(6) * u;
    };
    fac(ux, X0, X1);
    fac(uy, Y0, Y1);
    fac(uz, Z0, Z1);
    const R D2[3] = {R(6), R(-3), R(6)};   // psi'' (same on every axis)

    // contraction over z: T0/T1/T2[a][b] = sum_c mu w Z0/Z1/Z2
    R T0[3][3], T1[3][3], T2[3][3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) T0[aa][bb] = T1[aa][bb] = T2[aa][bb] = R(0);
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int aa = cx_of(i) + 1, bb = cy_of(i) + 1, cc = cz_of(i) + 1;
        const R mw = mu[i] * R(w_of(i));
        T0[aa][bb] += mw * Z0[cc];
        T1[aa][bb] += mw * Z1[cc];
        T2[aa][bb] += mw * D2[cc];
    });
    // over y
    R Y00[3], Y01[3], Y02[3], Y10[3], Y11[3], Y20[3];
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        Y00[aa] = Y01[aa] = Y02[aa] = Y10[aa] = Y11[aa] = Y20[aa] = R(0);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
            Y00[aa] += Y0[bb] * T0[aa][bb];
            Y01[aa] += Y0[bb] * T1[aa][bb];
            Y02[aa] += Y0[bb] * T2[aa][bb];
            Y10[aa] += Y1[bb] * T0[aa][bb];
            Y11[aa] += Y1[bb] * T1[aa][bb];
            Y20[aa] += D2[bb] * T0[aa][bb];
        }
    }
    // over x
    R K000 = 0, K001 = 0, K002 = 0, K010 = 0, K011 = 0, K020 = 0, K100 = 0, K101 = 0, K110 = 0, K200 = 0;
#pragma unroll
    for (int aa = 0; aa < 3; ++aa) {
        K000 += X0[aa] * Y00[aa];
        K001 += X0[aa] * Y01[aa];
        K002 += X0[aa] * Y02[aa];
        K010 += X0[aa] * Y10[aa];
        K011 += X0[aa] * Y11[aa];
        K020 += X0[aa] * Y20[aa];
        K100 += X1[aa] * Y00[aa];
        K101 += X1[aa] * Y01[aa];
        K110 += X1[aa] * Y10[aa];
        K200 += D2[aa] * Y00[aa];
    }
    // q_k = sum_j mu_j C_kj (columns of (M^T)^{-1})
    const R q4 = R(0.25) * (mu[7] + mu[10] - mu[8] - mu[9]);
    const R q5 = R(0.25) * (mu[11] + mu[14] - mu[12] - mu[13]);
    const R q6 = R(0.25) * (mu[15] + mu[18] - mu[16] - mu[17]);
    const R q7 = (mu[1] + mu[2] + mu[5] + mu[6]) * R(1.0 / 6.0) - (mu[3] + mu[4]) * R(1.0 / 3.0);
    const R q8 = (mu[1] + mu[2] + mu[3] + mu[4]) * R(1.0 / 6.0) - (mu[5] + mu[6]) * R(1.0 / 3.0);

    const R Arho = K000 + half * (gx * K100 + gy * K010 + gz * K001) +
                   om1 * (q4 * (-ux * uy + half * (gy * ux + gx * uy)) + q5 * (-ux * uz + half * (gz * ux + gx * uz)) +
                          q6 * (-uy * uz + half * (gz * uy + gy * uz)) + q7 * (-(ux * ux - uy * uy) + (gx * ux - gy * uy)) +
                          q8 * (-(ux * ux - uz * uz) + (gx * ux - gz * uz)));
    const R Aux = rho * (K100 + half * (gx * K200 + gy * K110 + gz * K101) +
                         om1 * (q4 * (-uy + half * gy) + q5 * (-uz + half * gz) + (q7 + q8) * (R(-2) * ux + gx)));
    const R Auy = rho * (K010 + half * (gx * K110 + gy * K020 + gz * K011) +
                         om1 * (q4 * (-ux + half * gx) + q6 * (-uz + half * gz) + q7 * (R(2) * uy - gy)));
    const R Auz = rho * (K001 + half * (gx * K101 + gy * K011 + gz * K002) +
                         om1 * (q5 * (-ux + half * gx) + q6 * (-uy + half * gy) + q8 * (R(2) * uz - gz)));
    const R irho = R(1) / rho;
    const R kap = sizeof(R) == 4 ? (R)j.kappa_f : (R)j.kappa;
    const R Bx = Aux * irho, By = Auy * irho;
    const R Bz = Auz * irho + (OBJ == LBM_J_UBULK ? kap * irho : R(0));
    const R vx = ux - half * gx, vy = uy - half * gy, vz = uz - half * gz;
    const R base = Arho - (Bx * vx + By * vy + Bz * vz);

    // lambda_i = base + c_i . B + (1 - omega)(cx cy q4 + cx cz q5 + cy cz q6 + (cx^2 - cy^2) q7
    // + (cx^2 - cz^2) q8), split into one term per axis and the three cross terms; only the
    // terms with a non-zero lattice coefficient are added
    const R o4 = om1 * q4, o5 = om1 * q5, o6 = om1 * q6, o7 = om1 * q7, o8 = om1 * q8;
    const R axm = (o7 + o8) - Bx, axp = (o7 + o8) + Bx;     // cx = -1, +1
    const R aym = -o7 - By, ayp = By - o7;
    const R azm = -o8 - Bz, azp = Bz - o8;
    R *lo = static_cast<R *>(j.lam);
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
        R l = base;
        if constexpr (cx == 1) l += axp;
        if constexpr (cx == -1) l += axm;
        if constexpr (cy == 1) l += ayp;
        if constexpr (cy == -1) l += aym;
        if constexpr (cz == 1) l += azp;
        if constexpr (cz == -1) l += azm;
        if constexpr (cx * cy == 1) l += o4;
        if constexpr (cx * cy == -1) l -= o4;
        if constexpr (cx * cz == 1) l += o5;
        if constexpr (cx * cz == -1) l -= o5;
        if constexpr (cy * cz == 1) l += o6;
        if constexpr (cy * cz == -1) l -= o6;
        lo[i * n + lc] = l;
    });

    // accumulators: objective, dJ/dg_z, dJ/domega
    jterm = R(0);
    if constexpr (OBJ == LBM_J_UBULK) {
        jterm = kap * uz;
    } else {
        // the wall is a cylinder, so (cx, cy, +1) and (cx, cy, -1) are wall links together:
        // their terms are summed as the difference f*(+1) - f*(-1), formed from the
        // closed-form differences psi(+1) - psi(-1) = 6 u_z and psi'(+1) - psi'(-1) = 6
        // (the rest weights cancel exactly instead of in floating point)
        if (p.nb != 0x1FFu) {
            const R dZ0 = R(6) * uz;
            sfor<0, 9>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int cx = k % 3 - 1, cy = k / 3 - 1;
                if constexpr (cx != 0 || cy != 0) {
                    constexpr int ip = dir_of(cx, cy, 1);
                    if (!dst_is_fluid<ip>(p)) {
                        const R x0y0 = X0[cx + 1] * Y0[cy + 1];
                        const R dP = x0y0 * dZ0;
                        const R dG = (gx * X1[cx + 1] * Y0[cy + 1] + gy * X0[cx + 1] * Y1[cy + 1]) * dZ0 +
                                     gz * x0y0 * R(6);
                        R dshear = 0;
                        if constexpr (cy == 0) dshear = R(cx) * R(0.5) * s5;
                        if constexpr (cx == 0) dshear = R(cy) * R(0.5) * s6;
                        jterm += wss * (R(w_of(ip)) * rho * (dP + half * dG) + om1 * dshear);
                    }
                }
            });
        }
    }
    const R gterm = half * rho * K001 + om1 * half * rho * (q5 * ux + q6 * uy - R(2) * q8 * uz) + half * Auz +
                    (OBJ == LBM_J_UBULK ? half * kap : R(0));
    wterm = -(q4 * s4 + q5 * s5 + q6 * s6 + q7 * s7 + q8 * s8);
    static_cast<R *>(j.acc_seg)[p.lc] += gterm;
}

// End of a segment of the reverse sweep: its dJ/dg_z sums join the FP64 totals (dense cells).
template <class R>
__global__ void k_flush_segment(const Member *members, R *acc_seg, double *acc) {
    const Member &d = members[0];
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= d.scells) return;
    const int z = (int)(s / d.Ps), r = (int)(s - (int64_t)z * d.Ps);
    const int4 ci = d.cellinfo[r];
    if (ci.x == -1) return;
    const int y = ci.x & 0xFFFF, x = (int)((uint32_t)ci.x >> 16);
    acc[((int64_t)z * d.ny + y) * d.nx + x] += (double)acc_seg[s];
    acc_seg[s] = R(0);
}

// One thread per ADJ_ZC consecutive planes of one stored position; the objective and
// dJ/domega terms are summed per warp in a fixed order and added to the warp's own FP64
// slots (deterministic), dJ/dg_z per cell.
template <int P, int OBJ>
__global__ void __launch_bounds__(256, LBM_ADJ_MIN_BLOCKS) k_adjoint(const __grid_constant__ StepArgs a,
                                                                     const AdjArgs j) {
    using R = typename Storage<P>::R;
    const Member &d = a.members[0];
    const uint32_t local = blockIdx.x * 256u + threadIdx.x;
    const uint32_t nzg = (uint32_t)(d.nz + ADJ_ZC - 1) / ADJ_ZC;
    R x0 = 0, x1 = 0;
    if (local < (uint32_t)d.Ps * nzg) {
        const uint32_t zg = fastdiv(local, d.ps_mul, d.ps_shr);
        const uint32_t r = local - zg * (uint32_t)d.Ps;
        CellPos p;
        if (cell_from_storage(d, zg * ADJ_ZC * (uint32_t)d.Ps + r, p)) {
#pragma unroll 1
            for (int k = 0; k < ADJ_ZC; ++k) {
                if (k > 0) {
                    if (p.z + 1 >= d.nz) break;
                    next_plane(d, p);
                }
                R y0, y1;
                adjoint_cell<P, OBJ>(a, j, d, p, y0, y1);
                x0 += y0;
                x1 += y1;
            }
        }
    }
    // warp sums of the objective and omega terms in the compute type, added to the
    // warp's own FP64 slots (fixed order, no block barrier)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 += __shfl_down_sync(0xFFFFFFFFu, x0, o);
        x1 += __shfl_down_sync(0xFFFFFFFFu, x1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        const int64_t wslot = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
        j.blockacc[wslot] += (double)x0;
        j.blockacc[(int64_t)j.nblocks * 8 + wslot] += (double)x1;
    }
}

// Column sums of up to five double arrays (stride n) into per-block partials.
static __global__ void __launch_bounds__(REDUCE_BLOCK) k_sum_columns(const double *base, int64_t n, int nv,
                                                                 double *partials) {
    __shared__ double sh[5 * 32];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if (k < nv) acc[k] += base[k * n + i];
    block_sum<5>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; ++k) partials[blockIdx.x * 5 + k] = acc[k];
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

template <int P, int BS, int MINB, int ZC = 1>
cudaError_t launch_step_shape(int wall, int parity, bool stats, const StepArgs &a, cudaStream_t s) {
    LBM_DISPATCH_WP(wall, parity, {
        if (stats) k_step<P, PA, W, EX_STATS, BS, MINB, MODEL_MRT_H6, ZC><<<a.nblocks_total, BS, 0, s>>>(a);
        else k_step<P, PA, W, EX_NONE, BS, MINB, MODEL_MRT_H6, ZC><<<a.nblocks_total, BS, 0, s>>>(a);
    });
    return cudaGetLastError();
}

template <int P, int BS, int MINB>
cudaError_t launch_step_pipe(int wall, int parity, bool stats, const StepArgs &a, cudaStream_t s) {
    using T = typename Storage<P>::T;
    const size_t smem = 2 * (size_t)Q * BS * sizeof(T);
    static int grid_cache[2][3][2] = {};            // resident blocks x SMs, per (parity, wall, stats)
    int &grid = grid_cache[parity][wall][stats ? 1 : 0];
    cudaError_t e = cudaSuccess;
    LBM_DISPATCH_WP(wall, parity, {
        auto kern = stats ? k_step_pipe<P, PA, W, EX_STATS, BS, MINB> : k_step_pipe<P, PA, W, EX_NONE, BS, MINB>;
        if (grid == 0) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            int per_sm = 0, dev = 0, sms = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem);
            if (e == cudaSuccess) e = cudaGetDevice(&dev);
            if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            grid = std::max(1, per_sm) * std::max(1, sms);
        }
        const int g = std::min(grid, a.nblocks_total);
        kern<<<g, BS, smem, s>>>(a);
    });
    return cudaGetLastError();
}

// The ablation models run in the default thread count of the precision with twice the
// registers of its shape (half the resident blocks): their populations stay live longer.
template <int P, int BS, int MINB>
cudaError_t launch_step_model(int wall, int parity, bool stats, const StepArgs &a, cudaStream_t s) {
    constexpr int MINB_R = MINB > 1 ? MINB / 2 : 1;
    LBM_DISPATCH_WP(wall, parity, {
        switch (a.collision) {
            case MODEL_BGK:
                if (stats) k_step<P, PA, W, EX_STATS, BS, MINB_R, MODEL_BGK><<<a.nblocks_total, BS, 0, s>>>(a);
                else k_step<P, PA, W, EX_NONE, BS, MINB_R, MODEL_BGK><<<a.nblocks_total, BS, 0, s>>>(a);
                break;
            case MODEL_O2:
                if (stats) k_step<P, PA, W, EX_STATS, BS, MINB_R, MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                else k_step<P, PA, W, EX_NONE, BS, MINB_R, MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                break;
            case MODEL_BGK | MODEL_O2:
                if (stats) k_step<P, PA, W, EX_STATS, BS, MINB_R, MODEL_BGK | MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                else k_step<P, PA, W, EX_NONE, BS, MINB_R, MODEL_BGK | MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                break;
            case MODEL_RATES:
                if (stats) k_step<P, PA, W, EX_STATS, BS, MINB_R, MODEL_RATES><<<a.nblocks_total, BS, 0, s>>>(a);
                else k_step<P, PA, W, EX_NONE, BS, MINB_R, MODEL_RATES><<<a.nblocks_total, BS, 0, s>>>(a);
                break;
            case MODEL_RATES | MODEL_O2:
                if (stats) k_step<P, PA, W, EX_STATS, BS, MINB_R, MODEL_RATES | MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                else k_step<P, PA, W, EX_NONE, BS, MINB_R, MODEL_RATES | MODEL_O2><<<a.nblocks_total, BS, 0, s>>>(a);
                break;
            default: return cudaErrorInvalidValue;
        }
    });
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_step(int wall, int parity, bool stats, const StepArgs &a, int variant, cudaStream_t s) {
    if (a.nblocks_total <= 0) return cudaSuccess;
    if (a.collision == MODEL_MRT_H6 && STEP_SHAPES[variant].staged)
        return launch_step_staged<P>(wall, parity, stats, a, variant, s);
    if (a.collision != MODEL_MRT_H6) {
        if constexpr (P == LBM_F64) return launch_step_model<P, 256, 2>(wall, parity, stats, a, s);
        else if constexpr (P == LBM_F32) return launch_step_model<P, 128, 8>(wall, parity, stats, a, s);
        else return cudaErrorInvalidValue;
    }
    if constexpr (P == LBM_F64) {
        return launch_step_shape<P, 256, 2>(wall, parity, stats, a, s);
    } else {
        switch (variant) {
            case 1: return launch_step_shape<P, 256, 3>(wall, parity, stats, a, s);
            case 2: return launch_step_shape<P, 128, 8>(wall, parity, stats, a, s);
            case 3: return launch_step_shape<P, 512, 2>(wall, parity, stats, a, s);
            case 4:
                if constexpr (P == LBM_F32) return launch_step_pipe<P, 256, 3>(wall, parity, stats, a, s);
                else return cudaErrorInvalidValue;
            case 5:
                if constexpr (P == LBM_F32) return launch_step_pipe<P, 128, 6>(wall, parity, stats, a, s);
                else return cudaErrorInvalidValue;
            case 6: return launch_step_shape<P, STEP_SHAPES[6].threads, STEP_SHAPES[6].min_blocks, STEP_SHAPES[6].zc>(wall, parity, stats, a, s);
            case 7: return launch_step_shape<P, STEP_SHAPES[7].threads, STEP_SHAPES[7].min_blocks, STEP_SHAPES[7].zc>(wall, parity, stats, a, s);
            case 8: return launch_step_shape<P, STEP_SHAPES[8].threads, STEP_SHAPES[8].min_blocks, STEP_SHAPES[8].zc>(wall, parity, stats, a, s);
            case 9: return launch_step_shape<P, STEP_SHAPES[9].threads, STEP_SHAPES[9].min_blocks, STEP_SHAPES[9].zc>(wall, parity, stats, a, s);
            case 10: return launch_step_shape<P, STEP_SHAPES[10].threads, STEP_SHAPES[10].min_blocks, STEP_SHAPES[10].zc>(wall, parity, stats, a, s);
            default: return launch_step_shape<P, 256, 4>(wall, parity, stats, a, s);
        }
    }
}

// Forward step of a single half-way pipe that also stores the adjoint moments (F32, F64).
template <int P>
cudaError_t launch_step_moments(int parity, const StepArgs &a, cudaStream_t s) {
    if constexpr (P == LBM_F64 || P == LBM_F32) {
        constexpr int BS = 256, MINB = (P == LBM_F64) ? 2 : 4;
        constexpr int ZC = (P == LBM_F64) ? 1 : STEP_SHAPES[MOM_VARIANT].zc;
        if (parity == 0) k_step<P, 0, LBM_HALFWAY, EX_MOMENTS, BS, MINB, MODEL_MRT_H6, ZC><<<a.nblocks_total, BS, 0, s>>>(a);
        else k_step<P, 1, LBM_HALFWAY, EX_MOMENTS, BS, MINB, MODEL_MRT_H6, ZC><<<a.nblocks_total, BS, 0, s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <int P>
cudaError_t launch_sum_columns(const double *base, int64_t n, int nv, double *partials, int n_partials_max,
                               double *out, cudaStream_t s) {
    int nb = (int)blocks_for(n, REDUCE_BLOCK);
    if (nb > n_partials_max) nb = n_partials_max;
    if (nb < 1) nb = 1;
    k_sum_columns<<<nb, REDUCE_BLOCK, 0, s>>>(base, n, nv, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, REDUCE_BLOCK, 0, s>>>(partials, nb, out);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_adjoint(const StepArgs &a, const AdjArgs &j, cudaStream_t s) {
    if constexpr (P == LBM_F64 || P == LBM_F32) {
        if (j.objective == LBM_J_UBULK) k_adjoint<P, LBM_J_UBULK><<<j.nblocks, 256, 0, s>>>(a, j);
        else k_adjoint<P, LBM_J_WSS><<<j.nblocks, 256, 0, s>>>(a, j);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
    }
}

template <int P>
cudaError_t launch_flush_segment(const StepArgs &a, const Member &hm, const AdjArgs &j, cudaStream_t s) {
    using R = typename Storage<P>::R;
    if constexpr (P == LBM_F64 || P == LBM_F32) {
        k_flush_segment<R><<<blocks_for(hm.scells, 256), 256, 0, s>>>(a.members, static_cast<R *>(j.acc_seg), j.acc);
        return cudaGetLastError();
    } else {
        return cudaErrorNotSupported;
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
    template cudaError_t launch_step_moments<P>(int, const StepArgs &, cudaStream_t);                    \
    template cudaError_t launch_adjoint<P>(const StepArgs &, const AdjArgs &, cudaStream_t);             \
    template cudaError_t launch_flush_segment<P>(const StepArgs &, const Member &, const AdjArgs &,       \
                                                 cudaStream_t);                                          \
    template cudaError_t launch_sum_columns<P>(const double *, int64_t, int, double *, int, double *,    \
                                               cudaStream_t);                                            \
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
