// lbm_staged.cuh -- the fused step with its loads staged in shared memory by bulk copies.
//
// In the compact layout the stored rows of a plane follow each other, so for a group of
// consecutive rows [y0, y1] of plane z the populations every direction needs form ONE
// contiguous, 64-byte aligned range per direction:
//   even step (own slots)  direction i: array i, plane z, rows [y0, y1];
//   odd step (pull)        direction i: array ibar, plane z - cz, rows [y0 - cy, y1 - cy]
// (the x - cx neighbours lie in the same rows).  A tile is (member, plane, row group).
// A persistent CTA walks over tiles.  Its last warp produces: for each tile, once the
// consumers have released the stage it goes into, one lane writes the tile's descriptor
// and issues 27 cp.async.bulk copies (global -> this CTA's shared memory, no multicast)
// plus one for the tile's 16-byte cell table, all completing on the stage's mbarrier.
// The other warps consume: they wait on that mbarrier (bounded), read their cells' 27
// populations from shared memory with addresses that need no per-direction arithmetic,
// collide, store straight to global memory and release the stage.  Loads are thus in
// flight without holding registers, and each population is still read once per step.
//
// Waits are bounded (about 2 s of the global timer): on expiry a warp records
// LBM_STAGED_TIMEOUT in a.err and returns (the producer first waits, bounded, for its
// copies in flight).
#pragma once

#include <algorithm>

#include "lbm_kernels.cuh"

namespace lbm {

constexpr int LBM_STAGED_TIMEOUT = 1;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits until phase `parity` of the mbarrier has completed, for about 2 s at most.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (global_ns() - t0 < 2000000000ull)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Bulk copy of `bytes` (a multiple of 16) from global memory into this CTA's shared
// memory (both addresses 16-byte aligned), completing on mbarrier `bar`.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Orders this thread's earlier generic-proxy accesses of shared memory before later
// async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Row group g of member d for staged shape `sel`: (y0, y1, lo[0], lo[1]), (lo[2], hi[0],
// hi[1], hi[2]) with lo[s] = rowbase(y0 + s - 1) and hi[s] = rowbase(y1 + s) (plane-local
// storage positions; rowbase(ny) = Ps): the rows shifted by s - 1 = -cy.
struct RowGroup { int y0, y1, lo[3], hi[3]; };
__device__ __forceinline__ RowGroup row_group(const Member &d, int sel, int g) {
    const int4 a = d.sg[sel][2 * g], b = d.sg[sel][2 * g + 1];
    RowGroup r;
    r.y0 = a.x; r.y1 = a.y;
    r.lo[0] = a.z; r.lo[1] = a.w; r.lo[2] = b.x;
    r.hi[0] = b.y; r.hi[1] = b.z; r.hi[2] = b.w;
    return r;
}

struct TileId { int m, z, g; };
__device__ __forceinline__ TileId tile_of(const StepArgs &a, int tile) {
    TileId t;
    t.m = find_member(a, tile);
    const Member &d = a.members[t.m];
    const int local = tile - a.block0[t.m];
    const int ng = d.nsg[a.sg_sel];
    t.z = local / ng;
    t.g = local - t.z * ng;
    return t;
}

// Shared-memory layout of one stage: 27 segments of `cap` storage elements (direction i
// at i * cap), then `cap` 16-byte cell-table entries.
template <class T>
__host__ __device__ constexpr uint32_t stage_bytes(int cap) {
    return (uint32_t)(27 * cap * (int)sizeof(T) + cap * 16);
}

// What the producer tells the consumers about the tile in a stage.
struct TileDesc { int m, z, lo[3], hi[3]; };

// The producer: the 28 bulk copies of tile `tile` into the stage at `stg`, completing on
// mbarrier `bar`, after writing the tile's descriptor (released to the consumers by the
// arrive on `bar`).
template <int P, int PAR>
__device__ __forceinline__ void issue_tile(const StepArgs &a, int tile, uint32_t stg, uint32_t bar, TileDesc *desc) {
    using T = typename Storage<P>::T;
    const TileId id = tile_of(a, tile);
    const Member &d = a.members[id.m];
    const RowGroup rg = row_group(d, a.sg_sel, id.g);
    desc->m = id.m;
    desc->z = id.z;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        desc->lo[s] = rg.lo[s];
        desc->hi[s] = rg.hi[s];
    }
    if (tile == a.skip_tile) return;          // failure-detection tests only: never completes
    const int cap = a.stage_cap;
    const T *base = static_cast<const T *>(a.pops) + d.off;
    const int64_t st = a.stride;
    uint32_t total = (uint32_t)(rg.hi[1] - rg.lo[1]) * 16u;
    if constexpr (PAR == 0) {
        total += 27u * (uint32_t)(rg.hi[1] - rg.lo[1]) * (uint32_t)sizeof(T);
    } else {
#pragma unroll
        for (int s = 0; s < 3; ++s) total += 9u * (uint32_t)(rg.hi[s] - rg.lo[s]) * (uint32_t)sizeof(T);
    }
    mbar_expect_tx(bar, total);
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        int arr, zz, s;
        if constexpr (PAR == 0) {
            arr = i; zz = id.z; s = 1;
        } else {
            arr = opp_of(i);
            zz = id.z - cz_of(i);
            zz = zz < 0 ? zz + d.nz : (zz >= d.nz ? zz - d.nz : zz);
            s = 1 - cy_of(i);
        }
        const uint32_t n = (uint32_t)(rg.hi[s] - rg.lo[s]);
        if (n > 0)
            bulk_load(stg + (uint32_t)(i * cap) * (uint32_t)sizeof(T),
                      base + (arr * st + (int64_t)zz * d.Ps + rg.lo[s]), n * (uint32_t)sizeof(T), bar);
    });
    bulk_load(stg + 27u * (uint32_t)cap * (uint32_t)sizeof(T), d.cellinfo + rg.lo[1],
              (uint32_t)(rg.hi[1] - rg.lo[1]) * 16u, bar);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

// Warp-specialised persistent kernel: warp NCW (the last) is the producer, warps
// 0..NCW-1 consume in NG groups of NCW / NG warps; group g takes the CTA's tiles k with
// k % NG == g, so NG tiles are worked on at once (a tile holds fewer cells than a full
// SM of threads, because shared memory bounds it).  Per stage a `full` mbarrier (one
// arrival with the copies' byte count) and an `empty` mbarrier (one arrival per warp of
// the consuming group once it has read the stage); no CTA-wide barrier inside the loop, so
// the consumer warps drift freely over the tiles.  Shared memory: STAGES stages of
// stage_bytes, then STAGES descriptors of 64 bytes, then the full and the empty mbarriers.
template <int P, int PAR, int WALL, int EXTRA, int NCW, int STAGES, int CTAS, int NG>
__global__ void __launch_bounds__((NCW + 1) * 32, CTAS) k_step_staged(const __grid_constant__ StepArgs a) {
    static_assert(NCW % NG == 0, "consumer warps split evenly into groups");
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const int cap = a.stage_cap;
    const uint32_t sb = stage_bytes<T>(cap);
    const uint32_t s0 = smem_addr(lbm_smem);
    TileDesc *descs = reinterpret_cast<TileDesc *>(lbm_smem + STAGES * sb);
    const uint32_t full0 = s0 + STAGES * sb + 64 * STAGES, empty0 = full0 + 8 * STAGES;
    const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, NCW / NG);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const int ntiles = a.nblocks_total;
    if (warp == NCW) {
        // ---- producer (one lane) ----
        if (lane != 0) return;
        int k = 0;
        bool ok = true;
        for (;; ++k) {
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile >= ntiles) break;
            const int s = k % STAGES;
            if (k >= STAGES && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)((k / STAGES - 1) & 1))) {
                ok = false;
                break;
            }
            fence_proxy_async();              // the consumers' reads of the stage come first
            issue_tile<P, PAR>(a, tile, s0 + s * sb, full0 + 8 * s, descs + s);
        }
        if (!ok) {
            atomicExch(a.err, LBM_STAGED_TIMEOUT);
            for (int j = (k > STAGES ? k - STAGES : 0); j < k; ++j)    // copies still in flight
                mbar_wait_bounded(full0 + 8 * (j % STAGES), (uint32_t)((j / STAGES) & 1));
        }
        return;
    }
    // ---- consumers ----
    const int64_t t = a.times ? a.times[a.tidx].t : a.t;
    const uint32_t st = (uint32_t)a.stride;
    const R inv = (R)a.f16_inv;
    constexpr bool RAW = raw_units<P, EXTRA, MODEL_MRT_H6>();
    constexpr int NC = NCW / NG * 32;                 // threads of a group
    const int group = warp / (NCW / NG);
    const int gtid = (int)threadIdx.x - group * NC;
    for (int k = group;; k += NG) {
        const int tile = blockIdx.x + k * gridDim.x;
        if (tile >= ntiles) break;
        const int stage = k % STAGES;
        if (!mbar_wait_bounded(full0 + 8 * stage, (uint32_t)((k / STAGES) & 1))) {
            atomicExch(a.err, LBM_STAGED_TIMEOUT);
            return;
        }
        const TileDesc td = descs[stage];
        const Member &d = a.members[td.m];
        const T *seg = reinterpret_cast<const T *>(lbm_smem + stage * sb);
        const int4 *sci = reinterpret_cast<const int4 *>(lbm_smem + stage * sb + 27 * cap * sizeof(T));
        const R stv = st_of<R>(a, td.m);
        const T *gbase = static_cast<const T *>(a.pops) + d.off;
        for (int r = td.lo[1] + gtid; r < td.hi[1]; r += NC) {
            const int4 ci = sci[r - td.lo[1]];
            if (ci.x == -1) continue;               // padding at the end of a row
            CellPos p;
            p.y = ci.x & 0xFFFF;
            p.x = (int)((uint32_t)ci.x >> 16);
            p.z = td.z;
            p.lc = (int32_t)(td.z * d.Ps + r);
            p.di = (td.z * d.ny + p.y) * d.nx + p.x;
            p.nb = (uint32_t)ci.y;
            p.ox[0] = -1; p.ox[1] = 0; p.ox[2] = 1;
            p.oy[0] = ci.z; p.oy[1] = 0; p.oy[2] = ci.w;
            p.oz[0] = td.z == 0 ? (d.nz - 1) * d.Ps : -d.Ps;
            p.oz[1] = 0;
            p.oz[2] = td.z == d.nz - 1 ? -(d.nz - 1) * d.Ps : d.Ps;
            R v[Q];
            if constexpr (PAR == 0) {
                const int q = r - td.lo[1];
                sfor<0, Q>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    v[i] = ld_pop<P, RAW>(seg + i * cap + q, inv);
                });
            } else {
                // source of direction i in its segment: rows shifted by -cy, x by -cx
                const int q0 = r - td.lo[1], qm = r + ci.z - td.lo[0], qp = r + ci.w - td.lo[2];
                if (p.nb == 0x1FFu) {
                    sfor<0, Q>([&](auto ic) {
                        constexpr int i = decltype(ic)::value;
                        constexpr int cy = cy_of(i);
                        const int q = (cy == 1 ? qm : (cy == -1 ? qp : q0)) - cx_of(i);
                        v[i] = ld_pop<P, RAW>(seg + i * cap + q, inv);
                    });
                } else {
                    // wall links read the cell's own slot (half-way bounce-back)
                    const uint32_t lc = (uint32_t)p.lc;
                    sfor<0, Q>([&](auto ic) {
                        constexpr int i = decltype(ic)::value;
                        constexpr int cy = cy_of(i);
                        const int q = (cy == 1 ? qm : (cy == -1 ? qp : q0)) - cx_of(i);
                        if constexpr (cx_of(i) == 0 && cy_of(i) == 0) {
                            v[i] = ld_pop<P, RAW>(seg + i * cap + q, inv);
                        } else {
                            const bool f = src_is_fluid<i>(p);
                            v[i] = f ? ld_pop<P, RAW>(seg + i * cap + (f ? q : 0), inv)
                                     : ld_pop<P, RAW>(gbase + (i * st + lc), inv);
                        }
                    });
                }
            }
            if constexpr (WALL == LBM_BOUZIDI) bouzidi_load_fix<R>(d, p, v);
            finish_cell<P, PAR, WALL, EXTRA, MODEL_MRT_H6>(a, d, p, t, stv, v);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * stage);
    }
}

// the staged kernels exist for the compact pipe layouts only (half-way and Bouzidi walls)
#define LBM_DISPATCH_STAGED(WALL_, PAR_, ...)                                      \
    do {                                                                          \
        if (WALL_ == LBM_HALFWAY) {                                               \
            if (PAR_ == 0) { constexpr int W = LBM_HALFWAY, PA = 0; __VA_ARGS__; } \
            else { constexpr int W = LBM_HALFWAY, PA = 1; __VA_ARGS__; }          \
        } else if (WALL_ == LBM_BOUZIDI) {                                        \
            if (PAR_ == 0) { constexpr int W = LBM_BOUZIDI, PA = 0; __VA_ARGS__; } \
            else { constexpr int W = LBM_BOUZIDI, PA = 1; __VA_ARGS__; }          \
        } else {                                                                  \
            return cudaErrorInvalidValue;                                         \
        }                                                                         \
    } while (0)

// Staged shape: persistent grid of (resident CTAs per SM) x SMs, at most one CTA per tile.
template <int P, int NCW, int STAGES, int CTAS, int NG>
struct StagedLaunch {
    static constexpr int BS = (NCW + 1) * 32;
    using T = typename Storage<P>::T;
    // per (parity, wall, statistics): configured dynamic shared memory and grid size
    static inline size_t smem_set[2][3][2] = {};
    static inline int grid[2][3][2] = {};

    template <class K>
    static cudaError_t configure(K kern, size_t smem, int pa, int w, int st) {
        if (smem_set[pa][w][st] == smem && grid[pa][w][st] > 0) return cudaSuccess;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, dev = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BS, smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        smem_set[pa][w][st] = smem;
        grid[pa][w][st] = per_sm * sms;
        return cudaSuccess;
    }

    static size_t smem_bytes(int cap) { return (size_t)STAGES * stage_bytes<T>(cap) + 80 * STAGES; }

    static cudaError_t prepare(int wall, int cap) {
        const size_t smem = smem_bytes(cap);
        cudaError_t e = cudaSuccess;
        for (int parity = 0; parity < 2 && e == cudaSuccess; ++parity)
            for (int st = 0; st < 2 && e == cudaSuccess; ++st) {
                LBM_DISPATCH_STAGED(wall, parity, {
                    e = st ? configure(k_step_staged<P, PA, W, EX_STATS, NCW, STAGES, CTAS, NG>, smem, PA, W, 1)
                           : configure(k_step_staged<P, PA, W, EX_NONE, NCW, STAGES, CTAS, NG>, smem, PA, W, 0);
                });
            }
        return e;
    }

    static cudaError_t launch(int wall, int parity, bool stats, const StepArgs &a, cudaStream_t s) {
        const size_t smem = smem_bytes(a.stage_cap);
        cudaError_t e = cudaSuccess;
        LBM_DISPATCH_STAGED(wall, parity, {
            auto kern = stats ? k_step_staged<P, PA, W, EX_STATS, NCW, STAGES, CTAS, NG>
                              : k_step_staged<P, PA, W, EX_NONE, NCW, STAGES, CTAS, NG>;
            e = configure(kern, smem, PA, W, stats ? 1 : 0);
            if (e != cudaSuccess) return e;
            const int g = std::min(grid[PA][W][stats ? 1 : 0], a.nblocks_total);
            kern<<<g, BS, smem, s>>>(a);
        });
        return cudaGetLastError();
    }
};

template <int P>
cudaError_t prepare_step(int wall, int variant) {
    const int k = staged_of(variant);
    if (k == 0)
        return StagedLaunch<P, STAGED_SHAPES[0].threads / 32 - 1, STAGED_SHAPES[0].stages,
                            STAGED_SHAPES[0].ctas_per_sm, STAGED_SHAPES[0].groups>::prepare(wall, staged_cap(P, 0));
    if (k == 1)
        return StagedLaunch<P, STAGED_SHAPES[1].threads / 32 - 1, STAGED_SHAPES[1].stages,
                            STAGED_SHAPES[1].ctas_per_sm, STAGED_SHAPES[1].groups>::prepare(wall, staged_cap(P, 1));
    return cudaSuccess;
}

template <int P>
cudaError_t launch_step_staged(int wall, int parity, bool stats, const StepArgs &a, int variant, cudaStream_t s) {
    if (STEP_SHAPES[variant].staged == 1)
        return StagedLaunch<P, STAGED_SHAPES[0].threads / 32 - 1, STAGED_SHAPES[0].stages,
                            STAGED_SHAPES[0].ctas_per_sm, STAGED_SHAPES[0].groups>::launch(wall, parity, stats, a, s);
    return StagedLaunch<P, STAGED_SHAPES[1].threads / 32 - 1, STAGED_SHAPES[1].stages,
                        STAGED_SHAPES[1].ctas_per_sm, STAGED_SHAPES[1].groups>::launch(wall, parity, stats, a, s);
}

}  // namespace lbm

// Explicit instantiation of the staged launchers for one storage precision.
#define LBM_INSTANTIATE_STAGED(P)                                                                       \
    namespace lbm {                                                                                     \
    template cudaError_t launch_step_staged<P>(int, int, bool, const StepArgs &, int, cudaStream_t);    \
    template cudaError_t prepare_step<P>(int, int);                                                     \
    }
