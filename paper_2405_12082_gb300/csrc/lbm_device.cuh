// lbm_device.cuh -- device building blocks of the D3Q27 MRT step.
//
// * Lattice (Appendix A): velocity order, opposite directions, weights.
// * Storage traits: populations are stored as f_i - w_i in double, float, half
//   (scaled by 2^s) or bfloat16; arithmetic runs in double or float.
// * The single-buffer AA access pattern: an even step reads and writes the cell's
//   own slots (slot i read as f_i, f*_i written to slot ibar); an odd step pulls
//   f_i from slot ibar of x - c_i and pushes f*_i to slot i of x + c_i.  Both touch
//   each slot exactly once, so the update is in place and race-free.  Wall links
//   (x - c_i solid) read and write the cell's own slot instead, which realises
//   half-way bounce-back; Bouzidi links add the interpolation of Eqs. (fbc1)-(fbc2)
//   on top of the same slots.
// * The collision of Eqs. (collision), (m*), (k*f*) in closed form.  With Lambda =
//   diag[1,1,1,1,omega x5,1 x18] every non-shear moment leaves the collision at
//   m^eq + R/2, so f* = f^eq + (1/2) g . grad_u f^eq + (1 - omega) sum_{k=4..8} C_k
//   (m_k - m_k^eq + R_k / 2), where C_k is column k of (M^T)^{-1} (nonzero only on
//   the 4 or 6 populations with the matching second-order velocity product).  The
//   sixth-order Hermite equilibrium factorises on D3Q27 as rho w_i psi(c_ix, u_x)
//   psi(c_iy, u_y) psi(c_iz, u_z), psi(0,u)/psi(0,0) = 1 - 3u^2/2 and
//   psi(+-1,u)/psi(+-1,0) = 1 +- 3u + 3u^2, which is what is evaluated.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>

#include "lbm.h"

namespace lbm {

// ---- lattice, Appendix A ----------------------------------------------------------
constexpr int Q = 27;
__host__ __device__ constexpr int cx_of(int i) {
    constexpr int v[27] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
    return v[i];
}
__host__ __device__ constexpr int cy_of(int i) {
    constexpr int v[27] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, 1, -1, -1, 1, 1, -1, -1};
    return v[i];
}
__host__ __device__ constexpr int cz_of(int i) {
    constexpr int v[27] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1};
    return v[i];
}
__host__ __device__ constexpr int opp_of(int i) {
    for (int j = 0; j < 27; ++j)
        if (cx_of(j) == -cx_of(i) && cy_of(j) == -cy_of(i) && cz_of(j) == -cz_of(i)) return j;
    return -1;
}
// Eq. (omegas): w0 = 8/27, w0/4 on faces, w0/16 on edges, w0/64 on corners.
__host__ __device__ constexpr double w_of(int i) {
    return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
}
// index of the velocity (cx, cy, cz)
__host__ __device__ constexpr int dir_of(int cx, int cy, int cz) {
    for (int j = 0; j < 27; ++j)
        if (cx_of(j) == cx && cy_of(j) == cy && cz_of(j) == cz) return j;
    return -1;
}
// in-plane neighbourhood bit of (cx, cy): bit (cy + 1) * 3 + (cx + 1)
__host__ __device__ constexpr int nbit(int cx, int cy) { return (cy + 1) * 3 + (cx + 1); }

template <int I, int N, class F>
__device__ __forceinline__ void sfor(F &&f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        sfor<I + 1, N>(f);
    }
}

// Row k of the moment basis of Eq. (Mmatrix) at velocity i: m_k = sum_i mt_coef(k, i) f_i.
__host__ __device__ constexpr int mt_coef(int k, int i) {
    const int x = cx_of(i), y = cy_of(i), z = cz_of(i);
    const int x2 = x * x, y2 = y * y, z2 = z * z;
    switch (k) {
        case 0: return 1;
        case 1: return x;
        case 2: return y;
        case 3: return z;
        case 4: return x * y;
        case 5: return x * z;
        case 6: return y * z;
        case 7: return x2 - y2;
        case 8: return x2 - z2;
        case 9: return x2 + y2 + z2;
        case 10: return x * y2 + x * z2;
        case 11: return x2 * y + y * z2;
        case 12: return x2 * z + y2 * z;
        case 13: return x * y2 - x * z2;
        case 14: return x2 * y - y * z2;
        case 15: return x2 * z - y2 * z;
        case 16: return x * y * z;
        case 17: return x2 * y2 + x2 * z2 + y2 * z2;
        case 18: return x2 * y2 + x2 * z2 - y2 * z2;
        case 19: return x2 * y2 - x2 * z2;
        case 20: return x2 * y * z;
        case 21: return x * y2 * z;
        case 22: return x * y * z2;
        case 23: return x * y2 * z2;
        case 24: return x2 * y * z2;
        case 25: return x2 * y2 * z;
        default: return x2 * y2 * z2;
    }
}

// (M^T)^{-1}, the back transform of Eq. (k*f*), by Gauss-Jordan elimination with
// partial pivoting, evaluated by the compiler: a[i][k] is the weight of moment k in
// population i.
struct MtInverse { double a[27][27]; };
constexpr MtInverse make_mt_inverse() {
    double A[27][54] = {};
    for (int k = 0; k < 27; ++k) {
        for (int i = 0; i < 27; ++i) A[k][i] = (double)mt_coef(k, i);
        A[k][27 + k] = 1.0;
    }
    for (int col = 0; col < 27; ++col) {
        int piv = col;
        for (int r = col + 1; r < 27; ++r) {
            const double a = A[r][col] < 0 ? -A[r][col] : A[r][col];
            const double b = A[piv][col] < 0 ? -A[piv][col] : A[piv][col];
            if (a > b) piv = r;
        }
        for (int j = 0; j < 54; ++j) {
            const double t = A[col][j];
            A[col][j] = A[piv][j];
            A[piv][j] = t;
        }
        const double d = A[col][col];
        for (int j = 0; j < 54; ++j) A[col][j] /= d;
        for (int r = 0; r < 27; ++r) {
            if (r == col || A[r][col] == 0.0) continue;
            const double fct = A[r][col];
            for (int j = 0; j < 54; ++j) A[r][j] -= fct * A[col][j];
        }
    }
    MtInverse out{};
    for (int i = 0; i < 27; ++i)
        for (int k = 0; k < 27; ++k) {
            const double v = A[i][27 + k];
            out.a[i][k] = (v < 1e-14 && v > -1e-14) ? 0.0 : v;    // exact zeros of the inverse
        }
    return out;
}
constexpr MtInverse kMtInv = make_mt_inverse();

// ---- storage ------------------------------------------------------------------------
// ld / st convert between the stored value and f - w; ldr / str move the stored value
// unscaled (the step kernels of the scaled half format work in units of 2^-s, see collide).
template <int P> struct Storage;
template <> struct Storage<LBM_F64> {
    using T = double; using R = double;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R ld(const T *p, R) { return *p; }
    static __device__ __forceinline__ void st(T *p, R v, R) { *p = v; }
    static __device__ __forceinline__ R ldr(const T *p) { return *p; }
    static __device__ __forceinline__ void str(T *p, R v) { *p = v; }
};
template <> struct Storage<LBM_F32> {
    using T = float; using R = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R ld(const T *p, R) { return *p; }
    static __device__ __forceinline__ void st(T *p, R v, R) { *p = v; }
    static __device__ __forceinline__ R ldr(const T *p) { return *p; }
    static __device__ __forceinline__ void str(T *p, R v) { *p = v; }
};
template <> struct Storage<LBM_F16S> {
    using T = __half; using R = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ R ld(const T *p, R inv_scale) { return __half2float(*p) * inv_scale; }
    static __device__ __forceinline__ void st(T *p, R v, R scale) { *p = __float2half_rn(v * scale); }
    static __device__ __forceinline__ R ldr(const T *p) { return __half2float(*p); }
    static __device__ __forceinline__ void str(T *p, R v) { *p = __float2half_rn(v); }
};
template <> struct Storage<LBM_BF16> {
    using T = __nv_bfloat16; using R = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R ld(const T *p, R) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void st(T *p, R v, R) { *p = __float2bfloat16_rn(v); }
    static __device__ __forceinline__ R ldr(const T *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ void str(T *p, R v) { *p = __float2bfloat16_rn(v); }
};

// ---- per-member description (host fills, device reads) ---------------------------------
// Storage layouts.  Dense: every cell of the box is stored, index (z ny + y) nx + x.
// Compact (pipes with half-way or Bouzidi walls): each row (y, z) stores only its run
// of fluid cells x0(y) .. x0(y) + span(y) - 1, starting on a 64-byte boundary; a plane
// holds Ps elements and cell (x, y, z) sits at z Ps + rowbase(y) + x - x0(y).  Solid
// cells have no storage (those walls never touch them), so every DRAM access atom
// carries fluid data except at the end of a row, and threads map onto stored cells only.
struct Member {
    int32_t nx, ny, nz, geometry;
    int64_t off;        // first stored cell of this member inside each population plane
    int64_t cells;      // nx * ny * nz
    int64_t scells;     // stored cells: cells (dense) or nz * Ps (compact)
    int64_t doff;       // first cell of this member in dense per-cell arrays (statistics)
    int32_t compact, Ps;
    uint32_t ps_mul, ps_shr;   // magic division by Ps
    const int32_t *rowbase;    // compact: [ny] start of row y inside a plane
    const int32_t *rowx0;      // compact: [ny] first fluid x of row y
    const uint16_t *rowof;     // compact: [Ps] row of each stored position (0xFFFF: padding)
    const int4 *cellinfo;      // compact: [Ps] per stored position: y | x << 16 (all ones:
                               // padding), the column's fluid mask, and the storage offsets
                               // of the rows y - 1 and y + 1 at the same x
    int64_t block0;     // first block of this member in a flat launch
    int64_t n_fluid;
    int64_t d2max;      // pipe: fluid iff (2x-nx+1)^2 + (2y-ny+1)^2 <= d2max
    double R, omega;
    double g[3];
    // trigger force, Eq. (TurbForce)
    int32_t trig, n_modes, kz, pad0;
    int32_t k_theta[LBM_MAX_TRIGGER_MODES];
    double amp[LBM_MAX_TRIGGER_MODES];     // h * A0 * weight
    double cph[LBM_MAX_TRIGGER_MODES], sph[LBM_MAX_TRIGGER_MODES];
    double kappa, l0, l, period;
    int64_t t_end;
    const void *gz_field;
    uint32_t nx_mul, nx_shr, ny_mul, ny_shr;   // magic division by nx and ny
    float gf[3], omegaf;       // float copies of g and omega for the FP32 kernels
    // general relaxation matrix Lambda = diag(lambda_k): 1 - lambda_k for k = 4..26
    // (k = 0..3 are conserved; read only by the general-rates collision)
    double om1k[23];
    float om1kf[23];
    const uint16_t *colmask;   // [ny][nx] in-plane 3x3 fluid mask of every column (device)
    const void *ftab;          // trigger: [3][ny][nx] column factors (P_x, P_y, P_z), compute type
    const void *ztab;          // trigger: [2][nz] cos, sin of kz 2 pi z / L, compute type
    const void *dtab;          // Bouzidi walls: [ny][nx][9][3] coefficients A, B, C of the link
                               // (cx, cy) at index nbit(cx, cy), compute type
    const int4 *sg[2];         // compact: row groups of the two staged launch shapes (2 int4
                               // per group, see lbm_staged.cuh), nsg[k] groups (0: shape
                               // not available for this member)
    int32_t nsg[2];
};

// Unsigned division by a fixed divisor d >= 1 for n < 2^31 (Granlund-Montgomery with
// a 31-bit dividend): l = ceil(log2 d), mul = ceil(2^(31+l) / d) < 2^32, and
// n / d = umulhi(n, mul) >> (l - 1).  d = 1 is flagged by shr = 0xFFFFFFFF.
inline void fastdiv_setup(uint32_t d, uint32_t &mul, uint32_t &shr) {
    if (d <= 1) { mul = 0; shr = 0xFFFFFFFFu; return; }
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;
    const uint64_t m = ((1ull << (31 + l)) + d - 1) / d;
    mul = (uint32_t)m;
    shr = l - 1;
}
__device__ __forceinline__ uint32_t fastdiv(uint32_t n, uint32_t mul, uint32_t shr) {
    return shr == 0xFFFFFFFFu ? n : (__umulhi(n, mul) >> shr);
}

// Per-step values for graph-captured chunks of steps: step index and sin(2 pi t / T) of
// every member's trigger (0 when off), filled by the host before each replay.
struct StepTime {
    int64_t t;
    double st[LBM_MAX_MEMBERS];
    float stf[LBM_MAX_MEMBERS];
};

struct StepArgs {
    void *pops;               // [27][stride] storage elements
    int64_t stride;           // cells per population plane (all members)
    const Member *members;    // device array
    int32_t n_members;
    int32_t nblocks_total;
    int64_t t;                // index of the step being taken
    float f16_scale, f16_inv;
    double *stats;            // [4][dstride] FP64 accumulators (sample steps), dense cells
    int64_t dstride;          // cells of all members in dense per-cell arrays
    double st[LBM_MAX_MEMBERS];      // sin(2 pi t / T) per member (0 when off)
    float stf[LBM_MAX_MEMBERS];      // the same in float for the FP32 kernels
    int32_t block0[LBM_MAX_MEMBERS + 1];
    const StepTime *times;    // when set, t and st come from times[tidx] (graph replays)
    int32_t tidx;
    void *moments;            // adjoint recompute: [9][cells] rho, u, s4..s8 of member 0
    int32_t collision;        // collision model (MODEL_* bits), the same for every member
    int32_t stage_cap;        // staged shapes: storage elements per direction segment
    int32_t sg_sel;           // staged shapes: which row-group table (0 or 1)
    int32_t *err;             // device status word (bounded waits that expired), or NULL
    int32_t skip_tile;        // failure-detection tests: a staged tile whose copies are never
                              // issued (its wait expires); -1 otherwise
};

__device__ __forceinline__ int find_member(const StepArgs &a, int blk) {
    int lo = 0, hi = a.n_members - 1;
    while (lo < hi) {          // largest m with block0[m] <= blk
        int mid = (lo + hi + 1) >> 1;
        if (a.block0[mid] <= blk) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---- geometry --------------------------------------------------------------------------
struct CellPos {
    int x, y, z;
    int32_t lc;              // storage index inside the member
    int32_t di;              // dense index (z ny + y) nx + x inside the member
    int32_t ox[3], oy[3], oz[3]; // neighbour offsets for c = -1, 0, +1 (periodic)
    uint32_t nb;             // in-plane fluid mask of the 3x3 neighbourhood
};

// Fluid test of a column (x, y) (pipe: distance to the axis < R, see lbm.h).
__host__ __device__ __forceinline__ bool col_fluid(const Member &d, int x, int y) {
    if (d.geometry == LBM_BOX) return true;
    const int64_t X = 2 * (int64_t)x - d.nx + 1, Y = 2 * (int64_t)y - d.ny + 1;
    return X * X + Y * Y <= d.d2max;
}

// Neighbour offsets (storage units) for c = -1, 0, +1 along x, y and z.
__device__ __forceinline__ void cell_offsets(const Member &d, CellPos &p) {
    if (!d.compact) {
        const int32_t nx = d.nx, nxy = d.nx * d.ny;
        p.ox[0] = p.x == 0 ? nx - 1 : -1;
        p.ox[1] = 0;
        p.ox[2] = p.x == nx - 1 ? -(nx - 1) : 1;
        p.oy[0] = p.y == 0 ? (d.ny - 1) * nx : -nx;
        p.oy[1] = 0;
        p.oy[2] = p.y == d.ny - 1 ? -(d.ny - 1) * nx : nx;
        p.oz[0] = p.z == 0 ? (d.nz - 1) * nxy : -nxy;
        p.oz[1] = 0;
        p.oz[2] = p.z == d.nz - 1 ? -(d.nz - 1) * nxy : nxy;
    } else {
        // rows of a pipe never reach the box edge: no x or y wrap.  A neighbour row
        // without fluid gets an unused offset (its cells are solid in the mask).
        const int32_t me = d.rowbase[p.y] - d.rowx0[p.y];
        p.ox[0] = -1;
        p.ox[1] = 0;
        p.ox[2] = 1;
        p.oy[0] = p.y > 0 ? (d.rowbase[p.y - 1] - d.rowx0[p.y - 1]) - me : 0;
        p.oy[1] = 0;
        p.oy[2] = p.y < d.ny - 1 ? (d.rowbase[p.y + 1] - d.rowx0[p.y + 1]) - me : 0;
        p.oz[0] = p.z == 0 ? (d.nz - 1) * d.Ps : -d.Ps;
        p.oz[1] = 0;
        p.oz[2] = p.z == d.nz - 1 ? -(d.nz - 1) * d.Ps : d.Ps;
    }
}

// Cell of storage index sidx (< scells) of member d.  Returns whether it is a fluid cell;
// for a compact padding slot nothing else is set.
__device__ __forceinline__ bool cell_from_storage(const Member &d, uint32_t sidx, CellPos &p) {
    if (!d.compact) {
        const uint32_t q = fastdiv(sidx, d.nx_mul, d.nx_shr);
        p.x = (int)(sidx - q * (uint32_t)d.nx);
        p.z = (int)fastdiv(q, d.ny_mul, d.ny_shr);
        p.y = (int)(q - (uint32_t)p.z * (uint32_t)d.ny);
        p.lc = (int32_t)sidx;
        p.di = (int32_t)sidx;
    } else {
        // one 16-byte table load gives position, fluid mask and row offsets, so the
        // neighbour addresses of the odd step wait on a single load
        p.z = (int)fastdiv(sidx, d.ps_mul, d.ps_shr);
        const int32_t r = (int32_t)(sidx - (uint32_t)p.z * (uint32_t)d.Ps);
        const int4 ci = d.cellinfo[r];
        if (ci.x == -1) return false;
        p.y = ci.x & 0xFFFF;
        p.x = (int)((uint32_t)ci.x >> 16);
        p.lc = (int32_t)sidx;
        p.di = (p.z * d.ny + p.y) * d.nx + p.x;
        p.nb = (uint32_t)ci.y;
        p.ox[0] = -1;
        p.ox[1] = 0;
        p.ox[2] = 1;
        p.oy[0] = ci.z;
        p.oy[1] = 0;
        p.oy[2] = ci.w;
        p.oz[0] = p.z == 0 ? (d.nz - 1) * d.Ps : -d.Ps;
        p.oz[1] = 0;
        p.oz[2] = p.z == d.nz - 1 ? -(d.nz - 1) * d.Ps : d.Ps;
        return (p.nb >> 4) & 1u;
    }
    p.nb = d.colmask[p.y * d.nx + p.x];
    cell_offsets(d, p);
    return (p.nb >> 4) & 1u;
}

// Cell of dense index di (< cells).  p.lc is the storage index of a fluid cell (every
// cell in the dense layout); returns whether the cell is fluid.
__device__ __forceinline__ bool cell_from_dense(const Member &d, uint32_t di, CellPos &p) {
    const uint32_t q = fastdiv(di, d.nx_mul, d.nx_shr);
    p.x = (int)(di - q * (uint32_t)d.nx);
    p.z = (int)fastdiv(q, d.ny_mul, d.ny_shr);
    p.y = (int)(q - (uint32_t)p.z * (uint32_t)d.ny);
    p.di = (int32_t)di;
    p.nb = d.colmask[p.y * d.nx + p.x];
    const bool fluid = (p.nb >> 4) & 1u;
    if (!d.compact) p.lc = (int32_t)di;
    else p.lc = fluid ? p.z * d.Ps + d.rowbase[p.y] + (p.x - d.rowx0[p.y]) : -1;
    cell_offsets(d, p);
    return fluid;
}

template <int I>
__device__ __forceinline__ int32_t nb_offset(const CellPos &p) {   // x + c_I
    return p.ox[cx_of(I) + 1] + p.oy[cy_of(I) + 1] + p.oz[cz_of(I) + 1];
}
template <int I>
__device__ __forceinline__ int32_t src_offset(const CellPos &p) {  // x - c_I
    return p.ox[1 - cx_of(I)] + p.oy[1 - cy_of(I)] + p.oz[1 - cz_of(I)];
}
template <int I>
__device__ __forceinline__ bool src_is_fluid(const CellPos &p) {
    return (p.nb >> nbit(-cx_of(I), -cy_of(I))) & 1u;
}
template <int I>
__device__ __forceinline__ bool dst_is_fluid(const CellPos &p) {
    return (p.nb >> nbit(cx_of(I), cy_of(I))) & 1u;
}

// ---- Bouzidi link coefficients, Eqs. (fbc1)-(fbc2) ---------------------------------------
// For a wall-pointing direction J of a fluid cell (x + c_J solid), the population
// returning in direction Jbar is A f*_J(x) + B f*_Jbar(x) + C f*_J(x - c_J).
template <class R>
struct BLink { R A, B, C; };

// The coefficients come from a per-column table filled on the host in FP64 from Delta,
// the fraction of the link from x to the circle r = R (the wall is a cylinder, so they
// depend on (x, y) and (cx, cy) only): Delta >= 1/2: A = 1 / (2 Delta), B = (2 Delta - 1) /
// (2 Delta), C = 0; Delta < 1/2 with x - c_J fluid: A = 2 Delta, B = 0, C = 1 - 2 Delta;
// otherwise the half-way values A = 1, B = C = 0.
template <class R, int J>
__device__ __forceinline__ BLink<R> bouzidi_link(const Member &d, const CellPos &p) {
    constexpr int cx = cx_of(J), cy = cy_of(J);
    const R *tab = static_cast<const R *>(d.dtab);
    const int64_t k = ((int64_t)(p.y * d.nx + p.x) * 9 + nbit(cx, cy)) * 3;
    return BLink<R>{tab[k], tab[k + 1], tab[k + 2]};
}

// The slot of a wall-pointing direction J holds A f*_J + B f*_Jbar of the previous step;
// the read of direction Jbar adds C f*_J(x - c_J), which is the value just read for J.
template <class R>
__device__ __forceinline__ void bouzidi_load_fix(const Member &d, const CellPos &p, R (&v)[27]) {
    if (p.nb == 0x1FFu) return;
    sfor<0, 27>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        if constexpr (cx_of(j) != 0 || cy_of(j) != 0) {
            if (!dst_is_fluid<j>(p)) {
                BLink<R> b = bouzidi_link<R, j>(d, p);
                v[opp_of(j)] += b.C * v[j];
            }
        }
    });
}

// ---- loading and storing the 27 populations of a cell ------------------------------------
// PAR 0: natural layout (after an odd step); PAR 1: reversed layout (after an even step).
// Slot of direction i read at a cell: PAR 0 -> (i, x); PAR 1 -> (ibar, x - c_i), or (i, x)
// across a wall link.  Slot written: PAR 0 -> (ibar, x); PAR 1 -> (i, x + c_i), or (ibar, x)
// across a wall link.  Wall links choose the address with a select, not a branch.
// Element indices are 32-bit: the library keeps 27 x stride below 2^32.
// RAW: the values stay in storage units (only the step kernels, see collide).
template <int P, bool RAW>
__device__ __forceinline__ typename Storage<P>::R ld_pop(const typename Storage<P>::T *q, typename Storage<P>::R inv) {
    if constexpr (RAW) return Storage<P>::ldr(q);
    else return Storage<P>::ld(q, inv);
}
template <int P, bool RAW>
__device__ __forceinline__ void st_pop(typename Storage<P>::T *q, typename Storage<P>::R v, typename Storage<P>::R sc) {
    if constexpr (RAW) Storage<P>::str(q, v);
    else Storage<P>::st(q, v, sc);
}

template <int P, int PAR, int WALL, bool RAW = false>
__device__ __forceinline__ void load_pops(const StepArgs &a, const Member &d, const CellPos &p,
                                          typename Storage<P>::R (&v)[Q]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    const T *base = static_cast<const T *>(a.pops) + d.off;
    const uint32_t st = (uint32_t)a.stride;
    const uint32_t lc = (uint32_t)p.lc;
    const R inv = (R)a.f16_inv;
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ib = opp_of(i);
        if constexpr (PAR == 0) {
            v[i] = ld_pop<P, RAW>(base + (i * st + lc), inv);
        } else {
            const uint32_t pull = ib * st + (uint32_t)(p.lc + src_offset<i>(p));
            if constexpr (WALL == LBM_FULLWAY || (cx_of(i) == 0 && cy_of(i) == 0)) {
                v[i] = ld_pop<P, RAW>(base + pull, inv);
            } else {
                const uint32_t own = i * st + lc;
                v[i] = ld_pop<P, RAW>(base + (src_is_fluid<i>(p) ? pull : own), inv);
            }
        }
    });
    if constexpr (WALL == LBM_BOUZIDI) bouzidi_load_fix<R>(d, p, v);
}

template <int P, int PAR, int WALL, bool RAW = false>
__device__ __forceinline__ void store_pops(const StepArgs &a, const Member &d, const CellPos &p,
                                           typename Storage<P>::R (&v)[Q]) {
    using S = Storage<P>;
    using T = typename S::T;
    using R = typename S::R;
    T *base = static_cast<T *>(a.pops) + d.off;
    const uint32_t st = (uint32_t)a.stride;
    const uint32_t lc = (uint32_t)p.lc;
    const R sc = (R)a.f16_scale;
    if constexpr (WALL == LBM_BOUZIDI) {
        // the value reflected into slot Jbar becomes A f*_J + B f*_Jbar
        if (p.nb != 0x1FFu) {
            R out[Q];
            sfor<0, Q>([&](auto ic) { constexpr int i = decltype(ic)::value; out[i] = v[i]; });
            sfor<0, Q>([&](auto jc) {
                constexpr int j = decltype(jc)::value;
                if constexpr (cx_of(j) != 0 || cy_of(j) != 0) {
                    if (!dst_is_fluid<j>(p)) {
                        BLink<R> b = bouzidi_link<R, j>(d, p);
                        out[j] = b.A * v[j] + b.B * v[opp_of(j)];
                    }
                }
            });
            sfor<0, Q>([&](auto ic) { constexpr int i = decltype(ic)::value; v[i] = out[i]; });
        }
    }
    sfor<0, Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        constexpr int ib = opp_of(i);
        if constexpr (PAR == 0) {
            st_pop<P, RAW>(base + (ib * st + lc), v[i], sc);
        } else {
            const uint32_t push = i * st + (uint32_t)(p.lc + nb_offset<i>(p));
            if constexpr (WALL == LBM_FULLWAY || (cx_of(i) == 0 && cy_of(i) == 0)) {
                st_pop<P, RAW>(base + push, v[i], sc);
            } else {
                const uint32_t own = ib * st + lc;
                st_pop<P, RAW>(base + (dst_is_fluid<i>(p) ? push : own), v[i], sc);
            }
        }
    });
}

// ---- acceleration g(x, t), Sec. II.B ----------------------------------------------------------
// The trigger force of Eq. (TurbForce) factorises into st(t) x z-factor x column factor:
// g_x = st cos(2 pi kz z / L) P_x(x, y), g_y = st cos(...) P_y(x, y),
// g_z = st sin(2 pi kz z / L) P_z(x, y); the column factors (zero outside the radial
// band) and the z factors are tabulated once per force by k_force_tables.
// Member parameters in the compute type (no FP64 arithmetic or conversion in FP32 kernels).
template <class R> __device__ __forceinline__ R g_of(const Member &d, int k) {
    if constexpr (sizeof(R) == 4) return d.gf[k]; else return d.g[k];
}
template <class R> __device__ __forceinline__ const R *lam1_of(const Member &d) {
    if constexpr (sizeof(R) == 4) return d.om1kf;
    else return d.om1k;
}
template <class R> __device__ __forceinline__ R omega_of(const Member &d) {
    if constexpr (sizeof(R) == 4) return d.omegaf; else return d.omega;
}
// sin(2 pi t / T) of member m for this step, in the compute type.
template <class R> __device__ __forceinline__ R st_of(const StepArgs &a, int m) {
    if constexpr (sizeof(R) == 4) return a.times ? a.times[a.tidx].stf[m] : a.stf[m];
    else return a.times ? a.times[a.tidx].st[m] : a.st[m];
}

template <class R>
__device__ __forceinline__ void acceleration(const Member &d, const CellPos &p, int64_t t, R st,
                                             R &gx, R &gy, R &gz) {
    gx = g_of<R>(d, 0);
    gy = g_of<R>(d, 1);
    gz = g_of<R>(d, 2);
    if (d.gz_field != nullptr) gz += static_cast<const R *>(d.gz_field)[p.di];
    if (d.trig && t < d.t_end) {
        const R *ft = static_cast<const R *>(d.ftab);
        const R *zt = static_cast<const R *>(d.ztab);
        const int32_t col = p.y * d.nx + p.x, ncol = d.nx * d.ny;
        const R sc = st * zt[p.z], ss = st * zt[d.nz + p.z];
        gx += sc * ft[col];
        gy += sc * ft[ncol + col];
        gz += ss * ft[2 * ncol + col];
    }
}

// Column and z factors of the trigger force (see acceleration), in double.
__device__ __forceinline__ void trigger_column(const Member &d, int x, int y, double &Px, double &Py, double &Pz) {
    Px = Py = Pz = 0.0;
    if (d.geometry != LBM_PIPE || !d.trig) return;
    const double px = 0.5 * (double)(2 * x - d.nx + 1), py = 0.5 * (double)(2 * y - d.ny + 1);
    const double r = sqrt(px * px + py * py);
    const double R = d.R, l0 = d.l0, l = d.l, L = (double)d.nz;
    if (!(r >= R - l0 - l && r <= R - l0 && r > 0.0)) return;
    const double ir = 1.0 / r, ct = px * ir, sn = py * ir;
    double sa, ca;
    sincospi(2.0 * (R - r - l0) / l, &sa, &ca);
    const double kz = (double)d.kz, kap = d.kappa;
    const double twopi = 6.283185307179586476925286766559;
    double Ar = 0, At = 0, Az = 0;
    for (int q = 0; q < d.n_modes; ++q) {
        const int kt = d.k_theta[q];
        double ck = 1, sk = 0;           // cos, sin of kt theta by repeated rotation
        for (int k = 0; k < kt; ++k) {
            const double c2 = ck * ct - sk * sn;
            sk = sk * ct + ck * sn;
            ck = c2;
        }
        const double cang = ck * d.cph[q] - sk * d.sph[q];
        const double sang = sk * d.cph[q] + ck * d.sph[q];
        const double A = d.amp[q];
        Ar += A * kap * (R * ir) * (kz * l / L) * (1.0 - ca) * cang;   // F_r = -st cz Ar
        At += A * (1.0 - kap) * (kz / kt) * (twopi * R / L) * sa * sang; // F_t =  st cz At
        Az += A * (R * ir) * sa * cang;                                 // F_z = -st sz Az
    }
    Px = -Ar * ct - At * sn;
    Py = -Ar * sn + At * ct;
    Pz = -Az;
}

// ---- collision ------------------------------------------------------------------------------
template <class R>
struct Macro { R drho, rho, ux, uy, uz; };

// The moments a collision needs, from v = f - w: drho = sum f - 1, j = sum c f and the raw
// second moments m4..m8 of Eq. (Mmatrix) (xy, xz, yz, x^2 - y^2, x^2 - z^2; the weights
// contribute nothing to them).  Every sum is formed from the z-triplets of the nine
// (cx, cy) columns of the lattice: P = f(+z) + f(-z), S = P + f(0), D = f(+z) - f(-z),
// which roughly halves the additions of summing each moment over its populations.
template <class R>
struct MomentSums { R drho, jx, jy, jz, m4, m5, m6, m7, m8; };

template <class R>
__device__ __forceinline__ MomentSums<R> moment_sums(const R (&v)[Q]) {
    R P[3][3], S[3][3], D[3][3];
    sfor<0, 9>([&](auto kc) {                       // column (cx, cy) = (a - 1, b - 1)
        constexpr int k = decltype(kc)::value, a = k % 3, b = k / 3;
        constexpr int ip = dir_of(a - 1, b - 1, 1), im = dir_of(a - 1, b - 1, -1), i0 = dir_of(a - 1, b - 1, 0);
        P[a][b] = v[ip] + v[im];
        S[a][b] = P[a][b] + v[i0];
        D[a][b] = v[ip] - v[im];
    });
    MomentSums<R> m;
    R Sa[3], Sb[3], Da[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Sa[k] = S[k][0] + S[k][1] + S[k][2];     // column sums at cx = k - 1
        Sb[k] = S[0][k] + S[1][k] + S[2][k];     // at cy = k - 1
        Da[k] = D[k][0] + D[k][1] + D[k][2];
    }
    m.drho = Sa[0] + Sa[1] + Sa[2];
    m.jx = Sa[2] - Sa[0];
    m.jy = Sb[2] - Sb[0];
    m.jz = Da[0] + Da[1] + Da[2];
    m.m4 = (S[2][2] - S[2][0]) - (S[0][2] - S[0][0]);
    m.m5 = Da[2] - Da[0];
    m.m6 = (D[0][2] - D[0][0]) + (D[1][2] - D[1][0]) + (D[2][2] - D[2][0]);
    m.m7 = (S[0][1] + S[2][1]) - (S[1][0] + S[1][2]);
    // x^2 - z^2: +1 on the cz = 0 populations of the cx != 0 columns, -1 on the cz != 0
    // populations of the cx = 0 columns
    constexpr int a0 = dir_of(-1, -1, 0), a1 = dir_of(-1, 0, 0), a2 = dir_of(-1, 1, 0);
    constexpr int b0 = dir_of(1, -1, 0), b1 = dir_of(1, 0, 0), b2 = dir_of(1, 1, 0);
    const R f0x = ((v[a0] + v[b0]) + (v[a1] + v[b1])) + (v[a2] + v[b2]);
    m.m8 = f0x - (P[1][0] + P[1][1] + P[1][2]);
    return m;
}

template <class R>
__device__ __forceinline__ Macro<R> macro_from_sums(const MomentSums<R> &s, R gx, R gy, R gz) {
    Macro<R> m;
    m.drho = s.drho;
    m.rho = R(1) + s.drho;
    const R ir = R(1) / m.rho;
    m.ux = s.jx * ir + R(0.5) * gx;
    m.uy = s.jy * ir + R(0.5) * gy;
    m.uz = s.jz * ir + R(0.5) * gz;
    return m;
}

template <class R>
__device__ __forceinline__ Macro<R> macroscopic(const R (&v)[Q], R gx, R gy, R gz) {
    return macro_from_sums<R>(moment_sums<R>(v), gx, gy, gz);
}

// One-axis factors of the product-form equilibrium (see the file header):
// dl[c+1] = psi_hat(c,u) - 1, hd[c+1] = (g/2) d psi_hat / du.
template <class R>
__device__ __forceinline__ void axis_factors(R u, R g, R (&dl)[3], R (&hd)[3]) {
    const R u2 = u * u;
    dl[1] = R(-1.5) * u2;
    dl[0] = R(3) * u2 - R(3) * u;
    dl[2] = R(3) * u2 + R(3) * u;
    const R hg = R(0.5) * g;
    hd[1] = hg * (R(-3) * u);
    hd[0] = hg * (R(6) * u - R(3));
    hd[2] = hg * (R(6) * u + R(3));
}

// Collision models: bit 0 selects the relaxation matrix (0: Lambda of Eq. (lambda);
// 1: Lambda = omega I, the single-relaxation-time operator of Eq. (srt) with the forcing
// term of Eq. (collision)), bit 1 the equilibrium (0: Eq. (BoltzmannEquilibriumDistribution);
// 1: its second-order truncation, the "LBM-O(2)" of Sec. III.B, with the forcing
// populations g . grad_u f^eq, which are Guo et al.'s (2002) for that equilibrium).
enum { MODEL_MRT_H6 = 0, MODEL_BGK = 1, MODEL_O2 = 2, MODEL_RATES = 4 };

// acc + e x for a lattice component e in {-1, 0, 1}; starting from -0 the sum is exact.
template <int E, class R> __device__ __forceinline__ R cterm(R acc, R x) {
    if constexpr (E == 1) return acc + x;
    else if constexpr (E == -1) return acc - x;
    else return acc;
}

// In-place collision of one fluid cell; v holds f - w on entry and f* - w on exit.
// With s_out, the five non-equilibrium shear moments s_k = m_k - m_k^eq + R_k / 2
// (k = 4..8) are returned as well (the adjoint stores them).
//
// Every model has the form f* = f^eq + F/2 + (1 - omega) N with F = g . grad_u f^eq:
// for the MRT, N = sum_{k=4..8} C_k s_k (the other moments relax with rate 1), and s_k
// is the same for both equilibria since they share their second moments and those of F;
// for the BGK, N = f - f^eq + F/2.  MODEL_RATES takes a general diagonal Lambda:
// f* = f^eq + F/2 + (M^T)^{-1} (1 - Lambda) M^T n with n = f - f^eq + F/2, whose moments
// 0..3 vanish (lam1[k - 4] = 1 - lambda_k).
//
// SCALED (default model only): v holds (f - w) sc on entry and leaves with (f* - w) sc,
// sc = 1 / inv a power of two (the half format's scale): the moment sums are taken in
// those units and multiplied by inv once, and sc enters the output constants, which is
// exact and saves the per-population scaling of loads and stores.
template <class R, int MODEL = MODEL_MRT_H6, bool SCALED = false>
__device__ __forceinline__ Macro<R> collide(R (&v)[Q], R gx, R gy, R gz, R omega, R *s_out = nullptr,
                                            const R *lam1 = nullptr, R inv = R(1), R sc = R(1)) {
    constexpr bool rates = (MODEL & MODEL_RATES) != 0;
    constexpr bool bgk = !rates && (MODEL & MODEL_BGK) != 0, o2 = (MODEL & MODEL_O2) != 0;
    static_assert(!SCALED || MODEL == MODEL_MRT_H6, "scaled units serve the default model only");
    MomentSums<R> ms = moment_sums<R>(v);
    if constexpr (SCALED) {
        ms.drho *= inv; ms.jx *= inv; ms.jy *= inv; ms.jz *= inv;
        ms.m4 *= inv; ms.m5 *= inv; ms.m6 *= inv; ms.m7 *= inv; ms.m8 *= inv;
    }
    const Macro<R> mm = macro_from_sums<R>(ms, gx, gy, gz);
    const R rho = mm.rho, ux = mm.ux, uy = mm.uy, uz = mm.uz;
    const R om1 = R(1) - omega;
    R s12 = 0, s34 = 0, s56 = 0, q4 = 0, q5 = 0, q6 = 0;
    R mk[23];                 // MODEL_RATES: moments 4..26 of n
#pragma unroll
    for (int k = 0; k < 23; ++k) mk[k] = 0;
    if constexpr (!bgk && !rates) {
        const R m4 = ms.m4, m5 = ms.m5, m6 = ms.m6, m7 = ms.m7, m8 = ms.m8;
        // (1 - omega)(m_k - m_k^eq + R_k / 2), k = 4..8, with the printed m^eq and R
        const R s4 = m4 - rho * ux * uy + R(0.5) * rho * (gy * ux + gx * uy);
        const R s5 = m5 - rho * ux * uz + R(0.5) * rho * (gz * ux + gx * uz);
        const R s6 = m6 - rho * uy * uz + R(0.5) * rho * (gz * uy + gy * uz);
        const R s7 = m7 - rho * (ux * ux - uy * uy) + rho * (gx * ux - gy * uy);
        const R s8 = m8 - rho * (ux * ux - uz * uz) + rho * (gx * ux - gz * uz);
        if (s_out) {
            s_out[0] = s4; s_out[1] = s5; s_out[2] = s6; s_out[3] = s7; s_out[4] = s8;
        }
        const R om1s = SCALED ? om1 * sc : om1;
        const R a4 = om1s * s4, a5 = om1s * s5, a6 = om1s * s6, a7 = om1s * s7, a8 = om1s * s8;
        s12 = (a7 + a8) * R(1.0 / 6.0);
        s34 = a8 * R(1.0 / 6.0) - a7 * R(1.0 / 3.0);
        s56 = a7 * R(1.0 / 6.0) - a8 * R(1.0 / 3.0);
        q4 = R(0.25) * a4;
        q5 = R(0.25) * a5;
        q6 = R(0.25) * a6;
    }
    const R drho = mm.drho;
    // post-collision value of population i from the equilibrium part pm1 = f^eq / (w rho) - 1
    // and frc = (1/2) g . grad_u (f^eq / (w rho))
    auto emit = [&](auto ic, R pm1, R frc) {
        constexpr int i = decltype(ic)::value;
        if constexpr (rates) {
            const R eq = R(w_of(i)) * (drho + rho * pm1), fh = R(w_of(i)) * rho * frc;
            const R ni = v[i] - eq + fh;
            sfor<4, Q>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr int cik = mt_coef(k, i);
                if constexpr (cik != 0) mk[k - 4] += R(cik) * ni;
            });
            v[i] = eq + fh;
        } else if constexpr (bgk) {
            const R eq = R(w_of(i)) * (drho + rho * pm1), fh = R(w_of(i)) * rho * frc;
            v[i] = eq + fh + om1 * (v[i] - eq + fh);
        } else {
            R f = R(w_of(i)) * (drho + rho * (pm1 + frc));
            if constexpr (i == 1 || i == 2) f += s12;
            if constexpr (i == 3 || i == 4) f += s34;
            if constexpr (i == 5 || i == 6) f += s56;
            if constexpr (i == 7 || i == 10) f += q4;
            if constexpr (i == 8 || i == 9) f -= q4;
            if constexpr (i == 11 || i == 14) f += q5;
            if constexpr (i == 12 || i == 13) f -= q5;
            if constexpr (i == 15 || i == 18) f += q6;
            if constexpr (i == 16 || i == 17) f -= q6;
            v[i] = f;
        }
    };
    if constexpr (!o2 && !bgk && !rates) {
        // the default model: f*_i - w_i = w_i drho + w_i rho (pm1 + frc) + shear term, with
        // pm1 + frc = Dxy + dz axy + Fxy (1 + dz) + hz axy = G + hz axy + dz H per (cx, cy)
        // column (G = Dxy + Fxy, H = axy + Fxy): three multiply-adds per population
        R dx[3], hx[3], dy[3], hy[3], dz[3], hz[3];
        axis_factors<R>(ux, gx, dx, hx);
        axis_factors<R>(uy, gy, dy, hy);
        axis_factors<R>(uz, gz, dz, hz);
        R G[3][3], H[3][3], A[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const R dxy = dx[a] + dy[b] + dx[a] * dy[b];
                const R axy = R(1) + dxy;
                const R fxy = hx[a] * (R(1) + dy[b]) + hy[b] * (R(1) + dx[a]);
                G[a][b] = dxy + fxy;
                H[a][b] = axy + fxy;
                A[a][b] = axy;
            }
        // w rho and w drho (plus the shear term of the population) per weight shell
        R w0 = R(w_of(0)), w1 = R(w_of(1)), w2 = R(w_of(7)), w3 = R(w_of(19));
        if constexpr (SCALED) {
            w0 *= sc; w1 *= sc; w2 *= sc; w3 *= sc;
        }
        const R wr0 = w0 * rho, wr1 = w1 * rho, wr2 = w2 * rho, wr3 = w3 * rho;
        const R wd0 = w0 * drho, wd1 = w1 * drho, wd2 = w2 * drho, wd3 = w3 * drho;
        const R c12 = wd1 + s12, c34 = wd1 + s34, c56 = wd1 + s56;
        const R c4p = wd2 + q4, c4m = wd2 - q4, c5p = wd2 + q5, c5m = wd2 - q5, c6p = wd2 + q6, c6m = wd2 - q6;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int a = cx_of(i) + 1, b = cy_of(i) + 1, c = cz_of(i) + 1;
            const R X = G[a][b] + hz[c] * A[a][b] + dz[c] * H[a][b];
            R wr, wd;
            if constexpr (i == 0) { wr = wr0; wd = wd0; }
            else if constexpr (i <= 6) {
                wr = wr1;
                wd = (i <= 2) ? c12 : ((i <= 4) ? c34 : c56);
            } else if constexpr (i <= 18) {
                wr = wr2;
                if constexpr (i == 7 || i == 10) wd = c4p;
                else if constexpr (i == 8 || i == 9) wd = c4m;
                else if constexpr (i == 11 || i == 14) wd = c5p;
                else if constexpr (i == 12 || i == 13) wd = c5m;
                else if constexpr (i == 15 || i == 18) wd = c6p;
                else wd = c6m;
            } else { wr = wr3; wd = wd3; }
            v[i] = wr * X + wd;
        });
    } else if constexpr (!o2) {
        R dx[3], hx[3], dy[3], hy[3], dz[3], hz[3];
        axis_factors<R>(ux, gx, dx, hx);
        axis_factors<R>(uy, gy, dy, hy);
        axis_factors<R>(uz, gz, dz, hz);
        // per (cx, cy) pair: Dxy = psi_x psi_y - 1 and the x/y force part
        R Dxy[3][3], Fxy[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                Dxy[a][b] = dx[a] + dy[b] + dx[a] * dy[b];
                Fxy[a][b] = hx[a] * (R(1) + dy[b]) + hy[b] * (R(1) + dx[a]);
            }
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int a = cx_of(i) + 1, b = cy_of(i) + 1, c = cz_of(i) + 1;
            const R dxy = Dxy[a][b];
            const R axy = R(1) + dxy;
            const R pm1 = dxy + dz[c] * axy;                       // psi_x psi_y psi_z - 1
            const R frc = Fxy[a][b] * (R(1) + dz[c]) + hz[c] * axy; // (1/2) g . grad psi
            emit(ic, pm1, frc);
        });
    } else {
        // second-order equilibrium: f^eq / (w rho) - 1 = 3 c.u + 9/2 (c.u)^2 - 3/2 u.u and
        // (1/2) g . grad_u of it = 3/2 (c.g - u.g) + 9/2 (c.u)(c.g)
        const R uu = ux * ux + uy * uy + uz * uz, ug = ux * gx + uy * gy + uz * gz;
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr int ex = cx_of(i), ey = cy_of(i), ez = cz_of(i);
            const R cu = cterm<ez>(cterm<ey>(cterm<ex>(R(-0.0), ux), uy), uz);
            const R cg = cterm<ez>(cterm<ey>(cterm<ex>(R(-0.0), gx), gy), gz);
            const R pm1 = R(3) * cu + R(4.5) * cu * cu - R(1.5) * uu;
            const R frc = R(1.5) * (cg - ug) + R(4.5) * cu * cg;
            emit(ic, pm1, frc);
        });
    }
    if constexpr (rates) {
#pragma unroll
        for (int k = 0; k < 23; ++k) mk[k] *= lam1[k];
        sfor<0, Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            R acc = v[i];
            sfor<4, Q>([&](auto kc) {
                constexpr int k = decltype(kc)::value;
                constexpr double aik = kMtInv.a[i][k];
                if constexpr (aik != 0.0) acc += R(aik) * mk[k - 4];
            });
            v[i] = acc;
        });
    }
    return mm;
}

}  // namespace lbm
