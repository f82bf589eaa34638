// lbm_api.cu -- the C ABI of include/lbm.h: contexts, validation, memory, launches.
#include <algorithm>
#include <array>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"

using lbm::Member;
using lbm::StepArgs;

cudaError_t lbm_launch_stats_profile(const double *acc, int64_t stride, const lbm::Member &d, double count, int nbins,
                                     double dr, double *bins, cudaStream_t s);

struct lbm_ctx {
    int precision = LBM_F32;
    int wall = LBM_HALFWAY;
    cudaStream_t stream = nullptr;
    std::vector<Member> hm;          // host copies of the member descriptors
    std::vector<lbm_grid> grids;
    std::vector<lbm_force> forces;
    Member *dm = nullptr;            // device copies
    int sel = 0;
    void *pops = nullptr;
    int64_t stride = 0;              // stored cells per population plane (all members)
    int64_t dense_total = 0;         // cells of all members in dense per-cell arrays
    std::vector<std::vector<int32_t>> rows;      // compact layout: rowbase[ny] ++ rowx0[ny] per member
    std::vector<std::vector<uint16_t>> rowof;    // compact layout: row of each stored position
    size_t esize = 0;                // bytes per stored population
    int64_t t = 0;
    float f16_scale = 1.f, f16_inv = 1.f;
    double *stats = nullptr;
    int32_t stats_every = 0;
    int64_t stats_count = 0;
    void *scratch = nullptr;         // staging for host buffers
    size_t scratch_bytes = 0;
    double *partials = nullptr;      // reduction partials + final (device)
    void *geo = nullptr;             // column masks and trigger tables of every member (device)
    int32_t *flags = nullptr;        // device status word of the step kernels (0 = fine)
    int32_t skip_tile = -1;          // lbm_test_expire_wait: tile of the next staged step left unissued
    int64_t check_every = 0;
    double max_drift = 0;
    std::vector<double> mass0;
    std::vector<bool> mass0_valid;
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    size_t ev_used = 0;
    std::vector<int64_t> ev_launches;   // step kernels covered by each timed event pair
    int64_t prof_launches_pending = 0;
    int64_t launches = 0;
    int variant = 0;                 // launch shape of the step kernel at even t
    int variant_odd = 0;             // ... and at odd t
    int collision = 0;               // collision model of the step kernel (lbm::MODEL_* bits)
    int model_bits = 0;              // lbm_set_collision: MODEL_BGK, MODEL_O2
    std::vector<bool> has_rates;     // per member: a general relaxation matrix was given
    std::vector<std::array<double, 27>> rates;
    // graph-captured chunks of steps
    int32_t graph_chunk = 0;
    cudaGraphExec_t gexec = nullptr;
    int gexec_variant = -1, gexec_variant_odd = -1, gexec_stats_every = -1;
    lbm::StepTime *d_times = nullptr;        // [graph_chunk] device table read by the graph
    lbm::StepTime *h_times[2] = {nullptr, nullptr};   // pinned staging, double-buffered
    cudaEvent_t h_done[2] = {nullptr, nullptr};
    int h_next = 0;
    // device allocator of this context (lbm_set_allocator at creation; NULL: cudaMalloc)
    lbm_alloc_fn alloc_fn = nullptr;
    lbm_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::string err;
};

namespace {

std::mutex g_alloc_mutex;
lbm_alloc_fn g_alloc_fn = nullptr;
lbm_free_fn g_free_fn = nullptr;
void *g_alloc_user = nullptr;

// Device memory of a context: the caller's allocator when one was set, else cudaMalloc.
// A hook result that is NULL or not 256-byte aligned counts as out of memory.
cudaError_t dev_alloc(lbm_ctx *c, void **p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 256;
    if (!c->alloc_fn) return cudaMalloc(p, bytes);
    void *q = c->alloc_fn(bytes, (void *)c->stream, c->alloc_user);
    if (!q) return cudaErrorMemoryAllocation;
    if (reinterpret_cast<uintptr_t>(q) % 256 != 0) {
        c->free_fn(q, (void *)c->stream, c->alloc_user);
        return cudaErrorMemoryAllocation;
    }
    *p = q;
    return cudaSuccess;
}

void dev_free(lbm_ctx *c, void *p) {
    if (!p) return;
    if (c->free_fn) c->free_fn(p, (void *)c->stream, c->alloc_user);
    else cudaFree(p);
}

}  // namespace

namespace {
thread_local std::string g_create_error;
}  // namespace

void lbm::set_thread_error(const char *msg) { g_create_error = msg ? msg : ""; }

namespace {

using lbm::default_variant;
using lbm::default_variant_odd;
using lbm::model_variant;

int set_err(lbm_ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_create_error = buf;
    return code;
}

int cuda_err(lbm_ctx *c, cudaError_t e, const char *what) {
    return set_err(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define LBM_CUDA(c, call)                                          \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_err((c), e_, #call);    \
    } while (0)

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// fluid iff (2x - nx + 1)^2 + (2y - ny + 1)^2 < 4 R^2  <=>  ... <= ceil(4 R^2) - 1
int64_t d2max_of(double R) { return (int64_t)std::ceil(4.0 * R * R) - 1; }

bool col_fluid_host(const Member &d, int x, int y) { return lbm::col_fluid(d, x, y); }

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Device tables of every member: the 3x3 in-plane fluid mask of each column and the
// trigger-force factors.  Allocated once; the force tables are refilled by set_force.
// Row groups of a compact member for the staged shapes: consecutive fluid rows [y0, y1]
// such that the rows shifted by -1, 0 and +1 each fit `cap` storage elements; per group
// two int4 (y0, y1, lo[0], lo[1]), (lo[2], hi[0], hi[1], hi[2]) with lo[s] =
// rowbase(y0 + s - 1), hi[s] = rowbase(y1 + s).  Empty when a single row does not fit.
std::vector<int4> row_groups(const Member &d, const std::vector<int32_t> &rows, int cap) {
    std::vector<int4> out;
    auto rb = [&](int y) { return y >= d.ny ? d.Ps : rows[y]; };
    auto span = [&](int y) { return rb(y + 1) - rb(y); };
    int first = -1, last = -1;
    for (int y = 0; y < d.ny; ++y)
        if (span(y) > 0) {
            if (first < 0) first = y;
            last = y;
        }
    if (first < 1 || last > d.ny - 2) return out;     // a pipe keeps a solid margin
    auto fits = [&](int y0, int y1) {
        for (int s = -1; s <= 1; ++s)
            if (rb(y1 + 1 + s) - rb(y0 + s) > cap) return false;
        return true;
    };
    for (int y = first; y <= last;) {
        if (!fits(y, y)) return std::vector<int4>();
        int y1 = y;
        while (y1 + 1 <= last && fits(y, y1 + 1)) ++y1;
        out.push_back(make_int4(y, y1, rb(y - 1), rb(y)));
        out.push_back(make_int4(rb(y + 1), rb(y1), rb(y1 + 1), rb(y1 + 2)));
        y = y1 + 1;
    }
    return out;
}

int build_tables(lbm_ctx *c) {
    const size_t es = c->precision == LBM_F64 ? 8 : 4;
    std::vector<size_t> at(c->hm.size() * 3), at_rows(c->hm.size()), at_delta(c->hm.size());
    std::vector<size_t> at_sg(c->hm.size() * 2);
    std::vector<std::vector<int4>> sg(c->hm.size() * 2);
    size_t total = 0;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        const Member &d = c->hm[m];
        const size_t ncol = (size_t)d.nx * d.ny;
        at_rows[m] = total;
        if (d.compact)
            total += align256(c->rows[m].size() * 4) + align256(c->rowof[m].size() * 2) +
                     align256(c->rowof[m].size() * sizeof(int4));
        at[3 * m] = total; total += align256(ncol * 2);
        at[3 * m + 1] = total; total += align256(3 * ncol * es);
        at[3 * m + 2] = total; total += align256(2 * (size_t)d.nz * es);
        at_delta[m] = total;
        if (c->wall == LBM_BOUZIDI) total += align256(27 * ncol * es);
        for (int k = 0; k < 2; ++k) {
            if (d.compact) sg[2 * m + k] = row_groups(d, c->rows[m], lbm::staged_cap(c->precision, k));
            at_sg[2 * m + k] = total;
            total += align256(sg[2 * m + k].size() * sizeof(int4));
        }
    }
    cudaError_t e = dev_alloc(c, &c->geo, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->geo = nullptr;
        return set_err(c, LBM_ENOMEM, "cannot allocate %zu bytes of geometry tables", total);
    }
    std::vector<uint16_t> mask;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        Member &d = c->hm[m];
        mask.assign((size_t)d.nx * d.ny, 0);
        for (int y = 0; y < d.ny; ++y)
            for (int x = 0; x < d.nx; ++x) {
                uint16_t nb = 0;
                for (int cy = -1; cy <= 1; ++cy)
                    for (int cx = -1; cx <= 1; ++cx)
                        if (col_fluid_host(d, x + cx, y + cy)) nb |= (uint16_t)(1u << lbm::nbit(cx, cy));
                mask[(size_t)y * d.nx + x] = nb;
            }
        char *g = (char *)c->geo;
        LBM_CUDA(c, cudaMemcpy(g + at[3 * m], mask.data(), mask.size() * 2, cudaMemcpyHostToDevice));
        d.colmask = (const uint16_t *)(g + at[3 * m]);
        if (d.compact) {
            const size_t rb = c->rows[m].size() * 4;
            LBM_CUDA(c, cudaMemcpy(g + at_rows[m], c->rows[m].data(), rb, cudaMemcpyHostToDevice));
            LBM_CUDA(c, cudaMemcpy(g + at_rows[m] + align256(rb), c->rowof[m].data(), c->rowof[m].size() * 2,
                                   cudaMemcpyHostToDevice));
            d.rowbase = (const int32_t *)(g + at_rows[m]);
            d.rowx0 = d.rowbase + d.ny;
            d.rowof = (const uint16_t *)(g + at_rows[m] + align256(rb));
            // per stored position: y | x << 16, fluid mask, offsets of rows y -/+ 1
            const std::vector<int32_t> &rw = c->rows[m];
            const std::vector<uint16_t> &ro = c->rowof[m];
            auto shift = [&](int y) { return rw[y] - rw[d.ny + y]; };   // rowbase - rowx0
            std::vector<int4> info(ro.size());
            for (size_t r = 0; r < ro.size(); ++r) {
                const int y = ro[r];
                if (y == 0xFFFF) { info[r] = make_int4(-1, 0, 0, 0); continue; }
                const int x = rw[d.ny + y] + ((int)r - rw[y]);
                const int me = shift(y);
                info[r] = make_int4((int)((uint32_t)y | ((uint32_t)x << 16)), mask[(size_t)y * d.nx + x],
                                    y > 0 ? shift(y - 1) - me : 0, y < d.ny - 1 ? shift(y + 1) - me : 0);
            }
            char *gi = g + at_rows[m] + align256(rb) + align256(ro.size() * 2);
            LBM_CUDA(c, cudaMemcpy(gi, info.data(), info.size() * sizeof(int4), cudaMemcpyHostToDevice));
            d.cellinfo = (const int4 *)gi;
        }
        for (int k = 0; k < 2; ++k) {
            const std::vector<int4> &grp = sg[2 * m + k];
            d.sg[k] = nullptr;
            d.nsg[k] = (int32_t)(grp.size() / 2);
            if (!grp.empty()) {
                LBM_CUDA(c, cudaMemcpy(g + at_sg[2 * m + k], grp.data(), grp.size() * sizeof(int4),
                                       cudaMemcpyHostToDevice));
                d.sg[k] = (const int4 *)(g + at_sg[2 * m + k]);
            }
        }
        d.ftab = g + at[3 * m + 1];
        d.ztab = g + at[3 * m + 2];
        d.dtab = nullptr;
        if (c->wall == LBM_BOUZIDI) {
            // Delta = (-b + sqrt(b^2 - a c)) / a of each link from a fluid column to a solid
            // one (a = |c|^2, b = p . c, c = |p|^2 - R^2, p relative to the axis), in double,
            // and the link coefficients A, B, C of Eqs. (fbc1)-(fbc2), stored in the compute
            // type (half-way values 1, 0, 0 where no second fluid point exists)
            std::vector<double> dl((size_t)27 * d.nx * d.ny, 0.0);
            for (int y = 0; y < d.ny; ++y)
                for (int x = 0; x < d.nx; ++x) {
                    if (!col_fluid_host(d, x, y)) continue;
                    const double px = 0.5 * (double)(2 * x - d.nx + 1), py = 0.5 * (double)(2 * y - d.ny + 1);
                    for (int cy = -1; cy <= 1; ++cy)
                        for (int cx = -1; cx <= 1; ++cx) {
                            if ((cx == 0 && cy == 0) || col_fluid_host(d, x + cx, y + cy)) continue;
                            const double a = (double)(cx * cx + cy * cy);
                            const double bb = px * cx + py * cy;
                            const double cc = px * px + py * py - d.R * d.R;
                            const double delta = (-bb + std::sqrt(bb * bb - a * cc)) / a;
                            double A = 1.0, B = 0.0, C = 0.0;
                            if (delta >= 0.5) {
                                A = 1.0 / (2.0 * delta);
                                B = (2.0 * delta - 1.0) / (2.0 * delta);
                            } else if (col_fluid_host(d, x - cx, y - cy)) {
                                A = 2.0 * delta;
                                C = 1.0 - 2.0 * delta;
                            }
                            double *t = &dl[(((size_t)y * d.nx + x) * 9 + lbm::nbit(cx, cy)) * 3];
                            t[0] = A;
                            t[1] = B;
                            t[2] = C;
                        }
                }
            char *gd = g + at_delta[m];
            if (es == 8) {
                LBM_CUDA(c, cudaMemcpy(gd, dl.data(), dl.size() * 8, cudaMemcpyHostToDevice));
            } else {
                std::vector<float> df(dl.begin(), dl.end());
                LBM_CUDA(c, cudaMemcpy(gd, df.data(), df.size() * 4, cudaMemcpyHostToDevice));
            }
            d.dtab = gd;
        }
    }
    return LBM_OK;
}

size_t esize_of(int p) {
    switch (p) {
        case LBM_F64: return 8;
        case LBM_F32: return 4;
        case LBM_F16S: return 2;
        case LBM_BF16: return 2;
    }
    return 0;
}

int check_force(lbm_ctx *c, const lbm_force *f) {
    if (!f) return LBM_OK;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(f->g[k])) return set_err(c, LBM_EINVAL, "force.g[%d] is not finite", k);
    if (f->trigger) {
        if (f->n_modes < 1 || f->n_modes > LBM_MAX_TRIGGER_MODES)
            return set_err(c, LBM_EINVAL, "force.n_modes must be in 1..%d", LBM_MAX_TRIGGER_MODES);
        for (int q = 0; q < f->n_modes; ++q)
            if (f->k_theta[q] < 1 || f->k_theta[q] > 64)
                return set_err(c, LBM_EINVAL, "force.k_theta[%d] must be in 1..64", q);
        if (!(f->period > 0)) return set_err(c, LBM_EINVAL, "force.period must be > 0");
        if (!(f->l > 0)) return set_err(c, LBM_EINVAL, "force.l must be > 0");
        if (!std::isfinite(f->A0) || !std::isfinite(f->kappa) || !std::isfinite(f->h) || !std::isfinite(f->l0))
            return set_err(c, LBM_EINVAL, "force trigger parameters must be finite");
    }
    return LBM_OK;
}

void fill_force(Member &d, const lbm_force *f) {
    for (int k = 0; k < 3; ++k) {
        d.g[k] = f ? f->g[k] : 0.0;
        d.gf[k] = (float)d.g[k];
    }
    d.trig = (f && f->trigger) ? 1 : 0;
    d.n_modes = d.trig ? f->n_modes : 0;
    d.kz = f ? f->kz : 0;
    for (int q = 0; q < LBM_MAX_TRIGGER_MODES; ++q) {
        const bool on = d.trig && q < d.n_modes;
        d.k_theta[q] = on ? f->k_theta[q] : 1;
        d.amp[q] = on ? f->h * f->A0 * f->weight[q] : 0.0;
        d.cph[q] = on ? std::cos(f->phase[q]) : 1.0;
        d.sph[q] = on ? std::sin(f->phase[q]) : 0.0;
    }
    d.kappa = f ? f->kappa : 0.0;
    d.l0 = f ? f->l0 : 0.0;
    d.l = f ? f->l : 1.0;
    d.period = (f && f->period > 0) ? f->period : 1.0;
    d.t_end = f ? f->t_end : 0;
    d.gz_field = f ? f->gz_field : nullptr;
}

int check_relax(lbm_ctx *c, const lbm_relax *r) {
    if (!(r->omega > 0.0 && r->omega < 2.0)) return set_err(c, LBM_EINVAL, "omega must be in (0, 2)");
    if (r->rates)
        for (int k = 0; k < 27; ++k)
            if (!(r->rates[k] >= 0.0 && r->rates[k] <= 2.0))
                return set_err(c, LBM_EINVAL, "relaxation rate %d must lie in [0, 2]", k);
    return LBM_OK;
}

// 1 - lambda_k (k = 4..26) of member d: the given rates, else Lambda of Eq. (lambda) or,
// for the BGK model, omega I.
void fill_lambda(Member &d, const double *rates, int model_bits) {
    for (int k = 4; k < 27; ++k) {
        const double lam = rates ? rates[k] : ((model_bits & lbm::MODEL_BGK) || k <= 8 ? d.omega : 1.0);
        d.om1k[k - 4] = 1.0 - lam;
        d.om1kf[k - 4] = (float)(1.0 - lam);
    }
}

void drop_graph(lbm_ctx *c);

// Recomputes every member's relaxation table and the step kernel's collision code; a new
// code returns the launch shape to the default and drops a captured graph.
int update_collision(lbm_ctx *c) {
    bool any = false;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        fill_lambda(c->hm[m], c->has_rates[m] ? c->rates[m].data() : nullptr, c->model_bits);
        any = any || c->has_rates[m];
    }
    const int code = any ? (lbm::MODEL_RATES | (c->model_bits & lbm::MODEL_O2)) : c->model_bits;
    if (code != 0 && c->precision != LBM_F32 && c->precision != LBM_F64)
        return set_err(c, LBM_EUNSUPPORTED, "the ablation collision models need F32 or F64 storage");
    if (code != c->collision) {
        c->collision = code;
        c->variant = code != 0 ? model_variant(c->precision) : default_variant(c->precision, c->wall);
        c->variant_odd = code != 0 ? model_variant(c->precision) : default_variant_odd(c->precision, c->wall);
        drop_graph(c);
    }
    return LBM_OK;
}

int build_member(lbm_ctx *c, const lbm_grid *g, const lbm_relax *r, const lbm_force *f, Member &d,
                 std::vector<int32_t> *rows = nullptr, std::vector<uint16_t> *rowof = nullptr) {
    if (!g || !r) return set_err(c, LBM_EINVAL, "grid and relax must not be NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1) return set_err(c, LBM_EINVAL, "grid sizes must be >= 1");
    const int64_t cells = (int64_t)g->nx * g->ny * g->nz;
    if (cells >= (1ll << 31)) return set_err(c, LBM_EINVAL, "a member may hold at most 2^31-1 cells");
    if (g->geometry != LBM_PIPE && g->geometry != LBM_BOX) return set_err(c, LBM_EINVAL, "unknown geometry");
    int rc = check_relax(c, r);
    if (rc) return rc;
    rc = check_force(c, f);
    if (rc) return rc;
    std::memset(&d, 0, sizeof d);
    d.nx = g->nx; d.ny = g->ny; d.nz = g->nz; d.geometry = g->geometry;
    d.cells = cells;
    d.R = g->R;
    d.omega = r->omega;
    d.omegaf = (float)r->omega;
    if (g->geometry == LBM_PIPE) {
        if (g->nx < 3 || g->ny < 3) return set_err(c, LBM_EINVAL, "a pipe needs nx, ny >= 3");
        if (!(g->R > 0.0) || !std::isfinite(g->R)) return set_err(c, LBM_EINVAL, "pipe radius must be > 0");
        d.d2max = d2max_of(g->R);
        for (int x = 0; x < g->nx; ++x)
            if (col_fluid_host(d, x, 0) || col_fluid_host(d, x, g->ny - 1))
                return set_err(c, LBM_EINVAL, "pipe must leave a solid margin at the box edge (R too large)");
        for (int y = 0; y < g->ny; ++y)
            if (col_fluid_host(d, 0, y) || col_fluid_host(d, g->nx - 1, y))
                return set_err(c, LBM_EINVAL, "pipe must leave a solid margin at the box edge (R too large)");
    }
    int64_t ncol = 0;
    for (int y = 0; y < g->ny; ++y)
        for (int x = 0; x < g->nx; ++x) ncol += col_fluid_host(d, x, y);
    d.n_fluid = ncol * g->nz;
    fill_force(d, f);
    lbm::fastdiv_setup((uint32_t)g->nx, d.nx_mul, d.nx_shr);
    lbm::fastdiv_setup((uint32_t)g->ny, d.ny_mul, d.ny_shr);
    // storage layout: compact fluid rows for pipes whose walls never touch solid cells
    // (positions are packed as 16-bit x and y)
    d.compact = (g->geometry == LBM_PIPE && g->wall != LBM_FULLWAY && rows && rowof && g->nx <= 0xFFFF &&
                 g->ny < 0xFFFF) ? 1 : 0;
    d.scells = d.cells;
    d.Ps = d.nx * d.ny;
    if (d.compact) {
        const int pad = (int)(64 / esize_of(g->precision));      // elements per 64 bytes
        rows->assign(2 * (size_t)g->ny, 0);
        int64_t ps = 0;
        for (int y = 0; y < g->ny; ++y) {
            int x0 = -1, x1 = -1;
            for (int x = 0; x < g->nx; ++x)
                if (col_fluid_host(d, x, y)) {
                    if (x0 < 0) x0 = x;
                    x1 = x;
                }
            (*rows)[y] = (int32_t)ps;
            (*rows)[g->ny + y] = x0 < 0 ? 0 : x0;
            if (x0 >= 0) ps += ((int64_t)(x1 - x0 + 1) + pad - 1) / pad * pad;
        }
        if (ps * g->nz >= (1ll << 31) || ps >= 0xFFFF * 64)
            return set_err(c, LBM_EINVAL, "pipe too large for the compact layout");
        rowof->assign((size_t)ps, 0xFFFF);
        for (int y = 0; y < g->ny; ++y)
            for (int x = 0; x < g->nx; ++x)
                if (col_fluid_host(d, x, y)) (*rowof)[(*rows)[y] + (x - (*rows)[g->ny + y])] = (uint16_t)y;
        d.Ps = (int32_t)ps;
        d.scells = ps * g->nz;
    }
    lbm::fastdiv_setup((uint32_t)std::max<int32_t>(d.Ps, 1), d.ps_mul, d.ps_shr);
    return LBM_OK;
}


// Launch shape of the step with index t.
int variant_at(const lbm_ctx *c, int64_t t) { return (t & 1) ? c->variant_odd : c->variant; }

StepArgs make_args(const lbm_ctx *c, int64_t t) {
    StepArgs a;
    std::memset(&a, 0, sizeof a);
    a.pops = c->pops;
    a.stride = c->stride;
    a.members = c->dm;
    a.n_members = (int32_t)c->hm.size();
    a.t = t;
    a.f16_scale = c->f16_scale;
    a.f16_inv = c->f16_inv;
    a.stats = c->stats;
    a.dstride = c->dense_total;
    a.collision = c->collision;
    const int v = variant_at(c, t);
    const int bs = lbm::step_threads(c->precision, v);
    const int zc = lbm::step_zc(c->precision, v);
    const int sk = lbm::staged_of(v);
    a.err = c->flags;
    a.skip_tile = -1;
    if (sk >= 0) {
        a.stage_cap = lbm::staged_cap(c->precision, sk);
        a.sg_sel = sk;
    }
    int64_t blk = 0;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        const Member &d = c->hm[m];
        a.st[m] = (d.trig && t < d.t_end) ? std::sin(2.0 * M_PI * (double)t / d.period) : 0.0;
        a.stf[m] = (float)a.st[m];
        a.block0[m] = (int32_t)blk;
        if (sk >= 0) {
            blk += (int64_t)d.nsg[sk] * d.nz;        // staged: one tile per (plane, row group)
        } else {
            // threads over (plane group, in-plane position); zc = 1 is every stored cell
            const int64_t work = (int64_t)d.Ps * ((d.nz + zc - 1) / zc);
            blk += (work + bs - 1) / bs;
        }
    }
    a.block0[c->hm.size()] = (int32_t)blk;
    a.nblocks_total = (int32_t)blk;
    a.times = nullptr;
    a.tidx = 0;
    return a;
}

void fill_times(const lbm_ctx *c, lbm::StepTime &st, int64_t t) {
    st.t = t;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        const Member &d = c->hm[m];
        st.st[m] = (d.trig && t < d.t_end) ? std::sin(2.0 * M_PI * (double)t / d.period) : 0.0;
        st.stf[m] = (float)st.st[m];
    }
}

int upload_members(lbm_ctx *c) {
    LBM_CUDA(c, cudaMemcpyAsync(c->dm, c->hm.data(), sizeof(Member) * c->hm.size(), cudaMemcpyHostToDevice,
                                c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int fill_force_tables(lbm_ctx *c, int m);

int ensure_scratch(lbm_ctx *c, size_t bytes) {
    if (bytes <= c->scratch_bytes) return LBM_OK;
    if (c->scratch) {
        cudaStreamSynchronize(c->stream);
        dev_free(c, c->scratch);
        c->scratch = nullptr;
        c->scratch_bytes = 0;
    }
    cudaError_t e = dev_alloc(c, &c->scratch, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, LBM_ENOMEM, "cannot allocate %zu bytes of staging memory", bytes);
    }
    c->scratch_bytes = bytes;
    return LBM_OK;
}

int prepare_variant(lbm_ctx *c);

int create_common(lbm_ctx **out, int32_t n, const lbm_grid *grids, const lbm_relax *relax,
                  const lbm_force *force, void *stream) {
    if (!out) return set_err(nullptr, LBM_EINVAL, "out must not be NULL");
    *out = nullptr;
    if (n < 1 || n > LBM_MAX_MEMBERS) return set_err(nullptr, LBM_EINVAL, "member count must be in 1..%d", LBM_MAX_MEMBERS);
    if (!grids || !relax) return set_err(nullptr, LBM_EINVAL, "grid and relax must not be NULL");
    const int prec = grids[0].precision, wall = grids[0].wall;
    if (esize_of(prec) == 0) return set_err(nullptr, LBM_EINVAL, "unknown precision %d", prec);
    if (wall != LBM_HALFWAY && wall != LBM_FULLWAY && wall != LBM_BOUZIDI)
        return set_err(nullptr, LBM_EINVAL, "unknown wall %d", wall);
    int s16 = grids[0].f16_log2_scale;
    if (s16 == 0) s16 = 16;
    if (s16 < 1 || s16 > 24) return set_err(nullptr, LBM_EINVAL, "f16_log2_scale must be in 1..24");
    lbm_ctx *c = new lbm_ctx();
    {
        std::lock_guard<std::mutex> lk(g_alloc_mutex);
        c->alloc_fn = g_alloc_fn;
        c->free_fn = g_free_fn;
        c->alloc_user = g_alloc_user;
    }
    c->precision = prec;
    c->wall = wall;
    c->variant = default_variant(prec, wall);
    c->variant_odd = lbm::default_variant_odd(prec, wall);
    c->stream = (cudaStream_t)stream;
    c->f16_scale = std::ldexp(1.0f, s16);
    c->f16_inv = std::ldexp(1.0f, -s16);
    c->hm.resize(n);
    int64_t off = 0, blk = 0, doff = 0;
    for (int k = 0; k < n; ++k) {
        if (grids[k].precision != prec || grids[k].wall != wall) {
            delete c;
            return set_err(nullptr, LBM_EINVAL, "all members must share precision and wall");
        }
        c->rows.emplace_back();
        c->rowof.emplace_back();
        int rc = build_member(nullptr, &grids[k], &relax[k], force ? &force[k] : nullptr, c->hm[k], &c->rows.back(),
                              &c->rowof.back());
        if (rc) { delete c; return rc; }
        c->hm[k].off = off;
        off += ceil_div(c->hm[k].scells, 64) * 64;   // keep every member 64-cell aligned
        c->hm[k].doff = doff;
        doff += ceil_div(c->hm[k].cells, 64) * 64;
        blk += ceil_div(c->hm[k].scells, 128);       // the smallest launch shape
        c->grids.push_back(grids[k]);
        c->has_rates.push_back(relax[k].rates != nullptr);
        c->rates.emplace_back();
        if (relax[k].rates) std::copy(relax[k].rates, relax[k].rates + 27, c->rates.back().begin());
        lbm_force fz;
        std::memset(&fz, 0, sizeof fz);
        c->forces.push_back(force ? force[k] : fz);
    }
    if (blk >= (1ll << 31)) { delete c; return set_err(nullptr, LBM_EINVAL, "grid too large"); }
    if (27 * off >= (1ll << 32)) {
        delete c;
        return set_err(nullptr, LBM_EUNSUPPORTED,
                       "27 x %lld cells exceed the 32-bit population index of the step kernels", (long long)off);
    }
    c->stride = off;
    c->dense_total = doff;
    c->esize = esize_of(prec);
    c->mass0.assign(n, 0.0);
    c->mass0_valid.assign(n, false);
    const size_t bytes = (size_t)27 * (size_t)c->stride * c->esize;
    cudaError_t e = dev_alloc(c, &c->pops, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return set_err(nullptr, LBM_ENOMEM, "cannot allocate %zu bytes of populations", bytes);
    }
    e = dev_alloc(c, (void **)&c->dm, sizeof(Member) * n);
    if (e == cudaSuccess) e = dev_alloc(c, (void **)&c->partials, sizeof(double) * (lbm::REDUCE_MAX_BLOCKS * 5 + 8));
    if (e == cudaSuccess) e = dev_alloc(c, (void **)&c->flags, 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->flags, 0, 256, c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbm_free(c);
        return set_err(nullptr, LBM_ENOMEM, "cannot allocate context buffers");
    }
    e = cudaMemsetAsync(c->pops, 0, bytes, c->stream);   // f - w = 0: rest state
    if (e != cudaSuccess) {
        lbm_free(c);
        return set_err(nullptr, LBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    int rc = update_collision(c);
    if (rc) {
        const std::string msg = c->err;
        lbm_free(c);
        return set_err(nullptr, rc, "%s", msg.c_str());
    }
    rc = build_tables(c);
    if (rc == LBM_OK) rc = upload_members(c);
    if (rc == LBM_OK) rc = prepare_variant(c);
    for (size_t m = 0; rc == LBM_OK && m < c->hm.size(); ++m) rc = fill_force_tables(c, (int)m);
    if (rc) {
        g_create_error = c->err;
        lbm_free(c);
        return rc;
    }
    *out = c;
    return LBM_OK;
}

template <class F>
int dispatch(lbm_ctx *c, F &&f) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (c->precision) {
        case LBM_F64: e = f(std::integral_constant<int, LBM_F64>{}); break;
        case LBM_F32: e = f(std::integral_constant<int, LBM_F32>{}); break;
        case LBM_F16S: e = f(std::integral_constant<int, LBM_F16S>{}); break;
        case LBM_BF16: e = f(std::integral_constant<int, LBM_BF16>{}); break;
    }
    if (e != cudaSuccess) return cuda_err(c, e, "kernel launch");
    c->launches++;
    return LBM_OK;
}

// Whether the context can run launch shape `variant`: a staged shape needs compact pipe
// members whose row groups fit its segments and the default collision model.
bool variant_available(const lbm_ctx *c, int variant) {
    if (!lbm::step_variant_ok(c->precision, variant)) return false;
    const int sk = lbm::staged_of(variant);
    if (sk < 0) return true;
    if (c->wall == LBM_FULLWAY || c->collision != 0) return false;
    for (const Member &d : c->hm)
        if (!d.compact || d.nsg[sk] < 1) return false;
    return true;
}

// Configures the kernels of the context's launch shape (shared-memory size of the staged
// kernels) ahead of any launch or graph capture.
int prepare_variant(lbm_ctx *c) {
    for (int v : {c->variant, c->variant_odd}) {
        if (lbm::staged_of(v) < 0) continue;
        cudaError_t e = cudaSuccess;
        switch (c->precision) {
            case LBM_F64: e = lbm::prepare_step<LBM_F64>(c->wall, v); break;
            case LBM_F32: e = lbm::prepare_step<LBM_F32>(c->wall, v); break;
            case LBM_F16S: e = lbm::prepare_step<LBM_F16S>(c->wall, v); break;
            default: e = lbm::prepare_step<LBM_BF16>(c->wall, v); break;
        }
        if (e != cudaSuccess) return cuda_err(c, e, "configuring the staged step kernels");
    }
    return LBM_OK;
}

int fill_force_tables(lbm_ctx *c, int m) {
    const Member &d = c->hm[m];
    if (!d.trig) return LBM_OK;
    void *ft = const_cast<void *>(d.ftab), *zt = const_cast<void *>(d.ztab);
    return dispatch(c, [&](auto P) {
        return lbm::launch_force_tables<decltype(P)::value>(c->dm, d, m, ft, zt, c->stream);
    });
}

int reduce_member(lbm_ctx *c, int m, double *host_out) {
    const StepArgs a = make_args(c, c->t);
    double *partials = c->partials, *dout = c->partials + lbm::REDUCE_MAX_BLOCKS * 5;
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_reduce<decltype(P)::value>(c->wall, (int)(c->t & 1), a, c->hm[m], m, partials,
                                                      lbm::REDUCE_MAX_BLOCKS, dout, c->stream);
    });
    if (rc) return rc;
    c->launches++;   // the final pass
    LBM_CUDA(c, cudaMemcpyAsync(host_out, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

// The step kernels' status word: a bounded wait that expired is reported once.
int check_flags(lbm_ctx *c) {
    int32_t f = 0;
    LBM_CUDA(c, cudaMemcpyAsync(&f, c->flags, sizeof f, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (f == 0) return LBM_OK;
    LBM_CUDA(c, cudaMemsetAsync(c->flags, 0, sizeof f, c->stream));
    return set_err(c, LBM_ETIMEOUT, "a step kernel's bounded wait for its staged tile expired (status %d)", f);
}

int stability_check(lbm_ctx *c) {
    int frc = check_flags(c);
    if (frc) return frc;
    for (size_t m = 0; m < c->hm.size(); ++m) {
        double r[5];
        int rc = reduce_member(c, (int)m, r);
        if (rc) return rc;
        if (r[4] > 0) return set_err(c, LBM_EUNSTABLE, "member %zu: %.0f cells with non-finite populations at t=%lld",
                                     m, r[4], (long long)c->t);
        if (!c->mass0_valid[m]) {
            c->mass0[m] = r[0];
            c->mass0_valid[m] = true;
        } else {
            const double drift = std::fabs(r[0] - c->mass0[m]) / (double)std::max<int64_t>(c->hm[m].n_fluid, 1);
            if (!(drift <= c->max_drift))
                return set_err(c, LBM_EUNSTABLE, "member %zu: relative mass drift %.3e above %.3e at t=%lld", m, drift,
                               c->max_drift, (long long)c->t);
        }
    }
    return LBM_OK;
}

int event_pair(lbm_ctx *c, cudaEvent_t &a, cudaEvent_t &b) {
    while (c->ev.size() < c->ev_used + 2) {
        cudaEvent_t e;
        LBM_CUDA(c, cudaEventCreate(&e));
        c->ev.push_back(e);
    }
    a = c->ev[c->ev_used];
    b = c->ev[c->ev_used + 1];
    c->ev_used += 2;
    c->ev_launches.push_back(0);
    return LBM_OK;
}

}  // namespace

// =====================================================================================
extern "C" {

int lbm_create(lbm_ctx **out, const lbm_grid *grid, const lbm_relax *relax, const lbm_force *force, void *stream) {
    return create_common(out, 1, grid, relax, force, stream);
}

int lbm_ensemble_create(lbm_ctx **out, int32_t n, const lbm_grid *grids, const lbm_relax *relax,
                        const lbm_force *force, void *stream) {
    return create_common(out, n, grids, relax, force, stream);
}

int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *user) {
    if ((alloc == nullptr) != (free_fn == nullptr)) {
        g_create_error = "lbm_set_allocator needs both hooks or neither";
        return LBM_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_alloc_mutex);
    g_alloc_fn = alloc;
    g_free_fn = free_fn;
    g_alloc_user = user;
    return LBM_OK;
}

void lbm_free(lbm_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    dev_free(c, c->pops);
    dev_free(c, c->dm);
    dev_free(c, c->stats);
    dev_free(c, c->scratch);
    dev_free(c, c->partials);
    dev_free(c, c->geo);
    dev_free(c, c->flags);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    dev_free(c, c->d_times);
    for (int b = 0; b < 2; ++b) {
        if (c->h_times[b]) cudaFreeHost(c->h_times[b]);
        if (c->h_done[b]) cudaEventDestroy(c->h_done[b]);
    }
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    cudaGetLastError();
    delete c;
}

const char *lbm_last_error(const lbm_ctx *c) {
    return c ? c->err.c_str() : g_create_error.c_str();
}

int lbm_set_stream(lbm_ctx *c, void *stream) {
    if (!c) return LBM_EINVAL;
    c->stream = (cudaStream_t)stream;
    return LBM_OK;
}

int lbm_select_member(lbm_ctx *c, int32_t m) {
    if (!c) return LBM_EINVAL;
    if (m < 0 || m >= (int32_t)c->hm.size()) return set_err(c, LBM_EINVAL, "member %d out of range", m);
    c->sel = m;
    return LBM_OK;
}

int lbm_get_info(lbm_ctx *c, lbm_info *info) {
    if (!c || !info) return LBM_EINVAL;
    const Member &d = c->hm[c->sel];
    info->n_cells = d.cells;
    info->n_fluid = d.n_fluid;
    info->t = c->t;
    info->population_bytes = (int64_t)27 * c->stride * (int64_t)c->esize;
    info->n_members = (int32_t)c->hm.size();
    info->precision = c->precision;
    info->launches = c->launches;
    info->variant = c->variant;
    info->variant_odd = c->variant_odd;
    info->step_threads = lbm::step_threads(c->precision, c->variant);
    info->n_variants = lbm::step_variants(c->precision);
    info->graph_chunk = c->graph_chunk;
    return LBM_OK;
}

int lbm_set_relax(lbm_ctx *c, const lbm_relax *r) {
    if (!c || !r) return LBM_EINVAL;
    int rc = check_relax(c, r);
    if (rc) return rc;
    const int m = c->sel;
    const bool had = c->has_rates[m];
    const double omega0 = c->hm[m].omega;
    const std::array<double, 27> rates0 = c->rates[m];
    c->hm[m].omega = r->omega;
    c->hm[m].omegaf = (float)r->omega;
    c->has_rates[m] = r->rates != nullptr;
    if (r->rates) std::copy(r->rates, r->rates + 27, c->rates[m].begin());
    rc = update_collision(c);
    if (rc) {                               // leave the member as it was
        c->hm[m].omega = omega0;
        c->hm[m].omegaf = (float)omega0;
        c->has_rates[m] = had;
        c->rates[m] = rates0;
        update_collision(c);
        return rc;
    }
    return upload_members(c);
}

int lbm_set_force(lbm_ctx *c, const lbm_force *f) {
    if (!c) return LBM_EINVAL;
    int rc = check_force(c, f);
    if (rc) return rc;
    fill_force(c->hm[c->sel], f);
    lbm_force fz;
    std::memset(&fz, 0, sizeof fz);
    c->forces[c->sel] = f ? *f : fz;
    rc = upload_members(c);
    if (rc) return rc;
    return fill_force_tables(c, c->sel);
}

int lbm_init(lbm_ctx *c, int32_t profile, double noise_amp, uint64_t seed) {
    if (!c) return LBM_EINVAL;
    if (profile != LBM_REST && profile != LBM_LAMINAR && profile != LBM_LOGLAW)
        return set_err(c, LBM_EINVAL, "unknown profile %d", profile);
    if (!std::isfinite(noise_amp)) return set_err(c, LBM_EINVAL, "noise_amp must be finite");
    for (size_t m = 0; m < c->hm.size(); ++m) {
        if (c->hm[m].geometry != LBM_PIPE && profile != LBM_REST)
            return set_err(c, LBM_EINVAL, "profiles other than REST need a pipe");
    }
    c->t = 0;
    LBM_CUDA(c, cudaMemsetAsync(c->pops, 0, (size_t)27 * c->stride * c->esize, c->stream));
    const StepArgs a = make_args(c, 0);
    for (size_t m = 0; m < c->hm.size(); ++m) {
        int rc = dispatch(c, [&](auto P) {
            return lbm::launch_init<decltype(P)::value>(c->wall, a, c->hm[m], (int)m, profile, noise_amp,
                                                        seed + (uint64_t)m, nullptr, nullptr, c->stream);
        });
        if (rc) return rc;
        c->mass0_valid[m] = false;
    }
    if (c->stats) {
        LBM_CUDA(c, cudaMemsetAsync(c->stats, 0, sizeof(double) * 4 * c->dense_total, c->stream));
        c->stats_count = 0;
    }
    return LBM_OK;
}

int lbm_init_fields(lbm_ctx *c, const double *rho, const double *u) {
    if (!c || !rho || !u) return LBM_EINVAL;
    const Member &d = c->hm[c->sel];
    const size_t n = (size_t)d.cells;
    const double *drho = rho, *du = u;
    const bool dev = is_device_ptr(rho) && is_device_ptr(u);
    if (!dev) {
        int rc = ensure_scratch(c, 4 * n * sizeof(double));
        if (rc) return rc;
        double *s = (double *)c->scratch;
        LBM_CUDA(c, cudaMemcpyAsync(s, rho, n * sizeof(double), cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaMemcpyAsync(s + n, u, 3 * n * sizeof(double), cudaMemcpyDefault, c->stream));
        drho = s;
        du = s + n;
    }
    if (c->t & 1) return set_err(c, LBM_EUNSUPPORTED, "lbm_init_fields resets t to 0; call it at even t");
    c->t = 0;
    const StepArgs a = make_args(c, 0);
    const int m = c->sel;
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_init<decltype(P)::value>(c->wall, a, c->hm[m], m, LBM_REST, 0.0, 0, drho, du, c->stream);
    });
    if (rc) return rc;
    c->mass0_valid[m] = false;
    if (!dev) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_test_expire_wait(lbm_ctx *c, int32_t tile) {
    if (!c) return LBM_EINVAL;
    if (lbm::staged_of(c->variant) < 0 && lbm::staged_of(c->variant_odd) < 0)
        return set_err(c, LBM_EUNSUPPORTED, "the current launch shapes have no staged tiles");
    if (tile < 0) return set_err(c, LBM_EINVAL, "tile must be >= 0");
    c->skip_tile = tile;
    return LBM_OK;
}

int lbm_set_check(lbm_ctx *c, int64_t every, double max_mass_drift) {
    if (!c) return LBM_EINVAL;
    if (every < 0 || !(max_mass_drift >= 0)) return set_err(c, LBM_EINVAL, "bad check parameters");
    c->check_every = every;
    c->max_drift = max_mass_drift;
    return LBM_OK;
}

}  // extern "C"

namespace {

// One step by a direct launch.
int step_direct(lbm_ctx *c) {
    const bool stats = c->stats && c->stats_every > 0 && (c->t % c->stats_every == 0);
    StepArgs a = make_args(c, c->t);
    if (c->skip_tile >= 0 && lbm::staged_of(variant_at(c, c->t)) >= 0) {
        a.skip_tile = c->skip_tile;
        c->skip_tile = -1;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
        int rc = event_pair(c, e0, e1);
        if (rc) return rc;
        LBM_CUDA(c, cudaEventRecord(e0, c->stream));
    }
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_step<decltype(P)::value>(c->wall, (int)(c->t & 1), stats, a, variant_at(c, c->t),
                                                    c->stream);
    });
    if (rc) return rc;
    if (c->prof) {
        LBM_CUDA(c, cudaEventRecord(e1, c->stream));
        c->ev_launches.back() += 1;
    }
    c->t++;
    if (stats) c->stats_count++;
    return LBM_OK;
}

void drop_graph(lbm_ctx *c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    c->gexec_variant = -1;
    c->gexec_variant_odd = -1;
    c->gexec_stats_every = -1;
}

// Captures graph_chunk steps that start at an even t (and, with statistics on, at a
// multiple of the statistics interval); every node reads its step index and trigger
// phase from d_times[k], so one instantiated graph serves every replay.
int build_graph(lbm_ctx *c) {
    drop_graph(c);
    int prc = prepare_variant(c);
    if (prc) return prc;
    const int every = (c->stats && c->stats_every > 0) ? c->stats_every : 0;
    cudaStream_t cs;
    LBM_CUDA(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_err(c, e, "cudaStreamBeginCapture");
    }
    // the two parities may run different launch shapes (block counts differ)
    StepArgs ap[2] = {make_args(c, 0), make_args(c, 1)};
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < c->graph_chunk && le == cudaSuccess; ++k) {
        StepArgs &a = ap[k & 1];
        a.times = c->d_times;
        a.tidx = k;
        const bool stats = every > 0 && (k % every == 0);
        const int v = variant_at(c, k);
        switch (c->precision) {
            case LBM_F64: le = lbm::launch_step<LBM_F64>(c->wall, k & 1, stats, a, v, cs); break;
            case LBM_F32: le = lbm::launch_step<LBM_F32>(c->wall, k & 1, stats, a, v, cs); break;
            case LBM_F16S: le = lbm::launch_step<LBM_F16S>(c->wall, k & 1, stats, a, v, cs); break;
            default: le = lbm::launch_step<LBM_BF16>(c->wall, k & 1, stats, a, v, cs); break;
        }
    }
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_err(c, le, "capture of the step chunk");
    }
    if (e != cudaSuccess) return cuda_err(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->gexec = nullptr;
        return cuda_err(c, e, "cudaGraphInstantiate");
    }
    c->gexec_variant = c->variant;
    c->gexec_variant_odd = c->variant_odd;
    c->gexec_stats_every = every;
    return LBM_OK;
}

// One replay of the captured chunk starting at the current (aligned) t.
int step_graph_chunk(lbm_ctx *c) {
    const int every = (c->stats && c->stats_every > 0) ? c->stats_every : 0;
    if (!c->gexec || c->gexec_variant != c->variant || c->gexec_variant_odd != c->variant_odd ||
        c->gexec_stats_every != every) {
        int rc = build_graph(c);
        if (rc) return rc;
    }
    const int b = c->h_next;
    c->h_next ^= 1;
    LBM_CUDA(c, cudaEventSynchronize(c->h_done[b]));   // staging buffer b is free again
    for (int k = 0; k < c->graph_chunk; ++k) fill_times(c, c->h_times[b][k], c->t + k);
    LBM_CUDA(c, cudaMemcpyAsync(c->d_times, c->h_times[b], sizeof(lbm::StepTime) * c->graph_chunk,
                                cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaEventRecord(c->h_done[b], c->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
        int rc = event_pair(c, e0, e1);
        if (rc) return rc;
        LBM_CUDA(c, cudaEventRecord(e0, c->stream));
    }
    LBM_CUDA(c, cudaGraphLaunch(c->gexec, c->stream));
    if (c->prof) {
        LBM_CUDA(c, cudaEventRecord(e1, c->stream));
        c->ev_launches.back() += c->graph_chunk;
    }
    c->launches += c->graph_chunk;
    if (every > 0) c->stats_count += (c->graph_chunk + every - 1) / every;
    c->t += c->graph_chunk;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_step(lbm_ctx *c, int64_t n) {
    if (!c) return LBM_EINVAL;
    if (n < 0) return set_err(c, LBM_EINVAL, "n must be >= 0");
    while (n > 0) {
        const int every = (c->stats && c->stats_every > 0) ? c->stats_every : 0;
        const int64_t t0 = c->t;
        const bool aligned = (c->t % 2 == 0) && (every == 0 || c->t % every == 0);
        int rc;
        int64_t done;
        if (c->graph_chunk > 0 && n >= c->graph_chunk && aligned) {
            rc = step_graph_chunk(c);
            done = c->graph_chunk;
        } else {
            rc = step_direct(c);
            done = 1;
        }
        if (rc) return rc;
        n -= done;
        if (c->check_every > 0 && (c->t / c->check_every) != (t0 / c->check_every)) {
            rc = stability_check(c);
            if (rc) return rc;
        }
    }
    return LBM_OK;
}

int lbm_set_graph(lbm_ctx *c, int32_t chunk) {
    if (!c) return LBM_EINVAL;
    if (chunk != 0 && (chunk < 2 || chunk > 4096 || (chunk & 1)))
        return set_err(c, LBM_EINVAL, "graph chunk must be 0 or an even number in 2..4096");
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graph(c);
    dev_free(c, c->d_times);
    c->d_times = nullptr;
    for (int b = 0; b < 2; ++b) {
        if (c->h_times[b]) cudaFreeHost(c->h_times[b]);
        c->h_times[b] = nullptr;
        if (c->h_done[b]) cudaEventDestroy(c->h_done[b]);
        c->h_done[b] = nullptr;
    }
    c->graph_chunk = 0;
    if (chunk == 0) return LBM_OK;
    const size_t bytes = sizeof(lbm::StepTime) * chunk;
    cudaError_t e = dev_alloc(c, (void **)&c->d_times, bytes);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        e = cudaMallocHost((void **)&c->h_times[b], bytes);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->h_done[b], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(c->h_done[b], c->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        lbm_set_graph(c, 0);
        return set_err(c, LBM_ENOMEM, "cannot allocate the step tables of the graph");
    }
    c->graph_chunk = chunk;
    return LBM_OK;
}

int lbm_set_variants(lbm_ctx *c, int32_t even, int32_t odd) {
    if (!c) return LBM_EINVAL;
    for (int variant : {even, odd}) {
        if (!lbm::step_variant_ok(c->precision, variant))
            return set_err(c, LBM_EINVAL, "launch-shape variant %d is not available for this storage (0..%d)", variant,
                           lbm::step_variants(c->precision) - 1);
        if (c->collision != 0 && variant != model_variant(c->precision))
            return set_err(c, LBM_EUNSUPPORTED, "the ablation collision models run in the default launch shape only");
        if (!variant_available(c, variant))
            return set_err(c, LBM_EUNSUPPORTED,
                           "launch shape %d (staged) needs pipes with half-way or Bouzidi walls whose rows fit %d "
                           "elements per segment",
                           variant, lbm::staged_cap(c->precision, std::max(0, lbm::staged_of(variant))));
    }
    const int old_even = c->variant, old_odd = c->variant_odd;
    c->variant = even;
    c->variant_odd = odd;
    const int rc = prepare_variant(c);
    if (rc) {
        c->variant = old_even;
        c->variant_odd = old_odd;
    }
    return rc;
}

int lbm_set_variant(lbm_ctx *c, int32_t variant) { return lbm_set_variants(c, variant, variant); }

int lbm_set_collision(lbm_ctx *c, int32_t model, int32_t equilibrium) {
    if (!c) return LBM_EINVAL;
    if ((model != LBM_MRT && model != LBM_BGK) || (equilibrium != LBM_EQ_HERMITE6 && equilibrium != LBM_EQ_ORDER2))
        return set_err(c, LBM_EINVAL, "unknown collision model %d / equilibrium %d", model, equilibrium);
    const int bits0 = c->model_bits;
    c->model_bits = (model == LBM_BGK ? lbm::MODEL_BGK : 0) | (equilibrium == LBM_EQ_ORDER2 ? lbm::MODEL_O2 : 0);
    int rc = update_collision(c);
    if (rc) {
        c->model_bits = bits0;
        update_collision(c);
        return rc;
    }
    return upload_members(c);
}

int lbm_autotune(lbm_ctx *c, int32_t steps, int32_t *variant, double *best_us) {
    if (!c) return LBM_EINVAL;
    if (steps < 2 || steps > 10000) return set_err(c, LBM_EINVAL, "steps must be in 2..10000");
    if (c->collision != 0)
        return set_err(c, LBM_EUNSUPPORTED, "the ablation collision models run in the default launch shape only");
    const int nv = lbm::step_variants(c->precision);
    const size_t bytes = (size_t)27 * c->stride * c->esize;
    void *save = nullptr;
    if (dev_alloc(c, &save, bytes) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, LBM_ENOMEM, "cannot allocate the state copy for autotuning");
    }
    LBM_CUDA(c, cudaMemcpyAsync(save, c->pops, bytes, cudaMemcpyDeviceToDevice, c->stream));
    const int64_t t_save = c->t, count_save = c->stats_count, launches_save = c->launches;
    double *stats_save = c->stats;
    const int64_t check_save = c->check_every;
    const bool prof_save = c->prof;
    c->stats = nullptr;          // no statistics, checks or profiling while tuning
    c->check_every = 0;
    c->prof = false;
    // one event before every timed step and one after the last: the even and the odd steps
    // are timed separately, so each parity gets its own fastest shape
    std::vector<cudaEvent_t> ev((size_t)steps + 1, nullptr);
    int rc = LBM_OK;
    for (size_t k = 0; k < ev.size() && rc == LBM_OK; ++k)
        if (cudaEventCreate(&ev[k]) != cudaSuccess) rc = cuda_err(c, cudaGetLastError(), "autotune events");
    int best[2] = {c->variant, c->variant_odd};
    double best_t[2] = {1e300, 1e300};
    for (int v = 0; v < nv && rc == LBM_OK; ++v) {
        if (!variant_available(c, v)) continue;
        c->variant = c->variant_odd = v;
        rc = prepare_variant(c);
        if (rc) break;
        c->t = t_save;
        for (int k = 0; k < 2 && rc == LBM_OK; ++k) rc = step_direct(c);
        if (rc) break;
        const int64_t t0 = c->t;
        for (int k = 0; k < steps && rc == LBM_OK; ++k) {
            cudaEventRecord(ev[k], c->stream);
            rc = step_direct(c);
        }
        cudaEventRecord(ev[steps], c->stream);
        if (cudaEventSynchronize(ev[steps]) != cudaSuccess) { rc = cuda_err(c, cudaGetLastError(), "autotune"); break; }
        double sum[2] = {0, 0};
        int cnt[2] = {0, 0};
        for (int k = 0; k < steps; ++k) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            const int par = (int)((t0 + k) & 1);
            sum[par] += 1e3 * ms;
            cnt[par] += 1;
        }
        for (int par = 0; par < 2; ++par) {
            const double us = cnt[par] ? sum[par] / cnt[par] : 1e300;
            if (us < best_t[par]) { best_t[par] = us; best[par] = v; }
        }
        cudaMemcpyAsync(c->pops, save, bytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    dev_free(c, save);
    c->t = t_save;
    c->stats = stats_save;
    c->stats_count = count_save;
    c->check_every = check_save;
    c->prof = prof_save;
    c->launches = launches_save;
    c->variant = best[0];
    c->variant_odd = best[1];
    if (rc == LBM_OK) rc = prepare_variant(c);
    const int best_v = best[0];
    const double best_us_pair = 0.5 * (best_t[0] + best_t[1]);
    if (rc) return rc;
    if (variant) *variant = best_v;
    if (best_us) *best_us = best_us_pair;
    return LBM_OK;
}

int lbm_moments(lbm_ctx *c, void *rho, void *u) {
    if (!c || !rho || !u) return LBM_EINVAL;
    const int m = c->sel;
    const Member &d = c->hm[m];
    const size_t es = c->precision == LBM_F64 ? 8 : 4;
    const size_t n = (size_t)d.cells;
    const bool dev = is_device_ptr(rho) && is_device_ptr(u);
    void *drho = rho, *du = u;
    if (!dev) {
        int rc = ensure_scratch(c, 4 * n * es);
        if (rc) return rc;
        drho = c->scratch;
        du = (char *)c->scratch + n * es;
    }
    const StepArgs a = make_args(c, c->t);
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_moments<decltype(P)::value>(c->wall, (int)(c->t & 1), a, d, m, drho, du, c->stream);
    });
    if (rc) return rc;
    if (!dev) {
        LBM_CUDA(c, cudaMemcpyAsync(rho, drho, n * es, cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaMemcpyAsync(u, du, 3 * n * es, cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx *c, double *f) {
    if (!c || !f) return LBM_EINVAL;
    const int m = c->sel;
    const Member &d = c->hm[m];
    const size_t bytes = (size_t)27 * d.cells * sizeof(double);
    const bool dev = is_device_ptr(f);
    double *df = f;
    if (!dev) {
        int rc = ensure_scratch(c, bytes);
        if (rc) return rc;
        df = (double *)c->scratch;
    }
    const StepArgs a = make_args(c, c->t);
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_get_pops<decltype(P)::value>(c->wall, (int)(c->t & 1), a, d, m, df, c->stream);
    });
    if (rc) return rc;
    if (!dev) {
        LBM_CUDA(c, cudaMemcpyAsync(f, df, bytes, cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx *c, const double *f) {
    if (!c || !f) return LBM_EINVAL;
    const int m = c->sel;
    const Member &d = c->hm[m];
    const size_t bytes = (size_t)27 * d.cells * sizeof(double);
    const bool dev = is_device_ptr(f);
    const double *df = f;
    if (!dev) {
        int rc = ensure_scratch(c, bytes);
        if (rc) return rc;
        LBM_CUDA(c, cudaMemcpyAsync(c->scratch, f, bytes, cudaMemcpyDefault, c->stream));
        df = (const double *)c->scratch;
    }
    const StepArgs a = make_args(c, c->t);
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_set_pops<decltype(P)::value>(c->wall, (int)(c->t & 1), a, d, m, df, c->stream);
    });
    if (rc) return rc;
    c->mass0_valid[m] = false;
    if (!dev) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_get_raw(lbm_ctx *c, void *buf, size_t bytes) {
    if (!c || !buf) return LBM_EINVAL;
    const size_t need = (size_t)27 * c->stride * c->esize;
    if (bytes != need) return set_err(c, LBM_EINVAL, "raw buffer must hold exactly %zu bytes", need);
    LBM_CUDA(c, cudaMemcpyAsync(buf, c->pops, need, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(buf)) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_set_raw(lbm_ctx *c, const void *buf, size_t bytes) {
    if (!c || !buf) return LBM_EINVAL;
    const size_t need = (size_t)27 * c->stride * c->esize;
    if (bytes != need) return set_err(c, LBM_EINVAL, "raw buffer must hold exactly %zu bytes", need);
    LBM_CUDA(c, cudaMemcpyAsync(c->pops, buf, need, cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(buf)) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LBM_OK;
}

int lbm_reduce(lbm_ctx *c, double *out) {
    if (!c || !out) return LBM_EINVAL;
    const int rc = reduce_member(c, c->sel, out);
    if (rc) return rc;
    return check_flags(c);
}

int lbm_stats_enable(lbm_ctx *c, int32_t every) {
    if (!c) return LBM_EINVAL;
    if (every < 1) return set_err(c, LBM_EINVAL, "stats interval must be >= 1");
    if (!c->stats) {
        cudaError_t e = dev_alloc(c, (void **)&c->stats, sizeof(double) * 4 * c->dense_total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->stats = nullptr;
            return set_err(c, LBM_ENOMEM, "cannot allocate statistics accumulators");
        }
    }
    LBM_CUDA(c, cudaMemsetAsync(c->stats, 0, sizeof(double) * 4 * c->dense_total, c->stream));
    c->stats_every = every;
    c->stats_count = 0;
    return LBM_OK;
}

int lbm_stats_get(lbm_ctx *c, double *acc, int64_t *count) {
    if (!c || !acc) return LBM_EINVAL;
    if (!c->stats) return set_err(c, LBM_EINVAL, "statistics are not enabled");
    const Member &d = c->hm[c->sel];
    LBM_CUDA(c, cudaMemcpy2DAsync(acc, (size_t)d.cells * sizeof(double), c->stats + d.doff,
                                  (size_t)c->dense_total * sizeof(double), (size_t)d.cells * sizeof(double), 4,
                                  cudaMemcpyDefault, c->stream));
    if (!is_device_ptr(acc)) LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (count) *count = c->stats_count;
    return LBM_OK;
}

int lbm_stats_profile(lbm_ctx *c, int32_t nbins, double dr, double *out) {
    if (!c || !out) return LBM_EINVAL;
    if (!c->stats || c->stats_count < 1) return set_err(c, LBM_EINVAL, "no statistics samples yet");
    if (nbins < 1 || nbins > 1024 || !(dr > 0)) return set_err(c, LBM_EINVAL, "need 1 <= nbins <= 1024 and dr > 0");
    const Member &d = c->hm[c->sel];
    if (d.geometry != LBM_PIPE) return set_err(c, LBM_EINVAL, "radial profiles need a pipe");
    int rc = ensure_scratch(c, sizeof(double) * 5 * nbins);
    if (rc) return rc;
    double *bins = (double *)c->scratch;
    LBM_CUDA(c, lbm_launch_stats_profile(c->stats + d.doff, c->dense_total, d, (double)c->stats_count, nbins, dr,
                                         bins, c->stream));
    c->launches++;
    std::vector<double> h(5 * (size_t)nbins);
    LBM_CUDA(c, cudaMemcpyAsync(h.data(), bins, sizeof(double) * 5 * nbins, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nbins; ++b) {
        const double n = h[5 * b];
        out[6 * b + 0] = (b + 0.5) * dr;
        out[6 * b + 1] = n;
        for (int k = 1; k < 5; ++k) out[6 * b + 1 + k] = n > 0 ? h[5 * b + k] / n : 0.0;
    }
    return LBM_OK;
}

int lbm_modes(lbm_ctx *c, const lbm_modes_cfg *cfg, double *E) {
    if (!c || !cfg || !E) return LBM_EINVAL;
    const int m = c->sel;
    const Member &d = c->hm[m];
    if (d.geometry != LBM_PIPE) return set_err(c, LBM_EINVAL, "modes need a pipe");
    if (cfg->n_sections < 1 || cfg->n_sections > d.nz) return set_err(c, LBM_EINVAL, "n_sections must be in 1..nz");
    if (cfg->n_rings < 1 || cfg->n_rings > 16) return set_err(c, LBM_EINVAL, "n_rings must be in 1..16");
    if (cfg->n_theta < 8 || cfg->n_theta > 4096) return set_err(c, LBM_EINVAL, "n_theta must be in 8..4096");
    if (cfg->n_modes < 0 || cfg->n_modes >= cfg->n_theta) return set_err(c, LBM_EINVAL, "n_modes must be in 0..n_theta-1");
    lbm::ModesArgs ma;
    std::memset(&ma, 0, sizeof ma);
    ma.n_sections = cfg->n_sections;
    ma.n_rings = cfg->n_rings;
    ma.n_theta = cfg->n_theta;
    ma.n_modes = cfg->n_modes;
    for (int j = 0; j < cfg->n_rings; ++j) {
        const double rr = cfg->r_over_R[j];
        if (!(rr > 0.0) || rr * d.R + 1.5 >= 0.5 * std::min(d.nx, d.ny))
            return set_err(c, LBM_EINVAL, "ring %d: r_over_R must put the ring inside the box", j);
        ma.r_over_R[j] = rr;
    }
    const size_t bytes = sizeof(double) * cfg->n_sections * cfg->n_rings * (cfg->n_modes + 1);
    const bool dev = is_device_ptr(E);
    double *dE = E;
    if (!dev) {
        int rc = ensure_scratch(c, bytes);
        if (rc) return rc;
        dE = (double *)c->scratch;
    }
    const StepArgs a = make_args(c, c->t);
    int rc = dispatch(c, [&](auto P) {
        return lbm::launch_modes<decltype(P)::value>(c->wall, (int)(c->t & 1), a, d, m, ma, dE, c->stream);
    });
    if (rc) return rc;
    if (!dev) {
        LBM_CUDA(c, cudaMemcpyAsync(E, dE, bytes, cudaMemcpyDefault, c->stream));
        LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return LBM_OK;
}

int lbm_adjoint(lbm_ctx *c, int64_t T, int32_t objective, int64_t checkpoint_every, double *J, double *dJ_dgz,
                double *dJ_domega) {
    if (!c) return LBM_EINVAL;
    if (T < 1) return set_err(c, LBM_EINVAL, "T must be >= 1");
    if (objective != LBM_J_UBULK && objective != LBM_J_WSS) return set_err(c, LBM_EINVAL, "unknown objective");
    if (checkpoint_every < 0) return set_err(c, LBM_EINVAL, "checkpoint_every must be >= 0");
    if (c->hm.size() != 1 || c->wall != LBM_HALFWAY || (c->precision != LBM_F32 && c->precision != LBM_F64) ||
        c->hm[0].geometry != LBM_PIPE)
        return set_err(c, LBM_EUNSUPPORTED, "the adjoint needs a single half-way pipe in F32 or F64 storage");
    if (c->collision != 0)
        return set_err(c, LBM_EUNSUPPORTED, "the adjoint is derived for the MRT model with the Hermite equilibrium");
    if (c->hm[0].trig) return set_err(c, LBM_EUNSUPPORTED, "the adjoint takes no trigger force");
    const Member &d = c->hm[0];
    const int64_t K = checkpoint_every > 0 ? std::min<int64_t>(checkpoint_every, T)
                                           : std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)T)));
    const int64_t nseg = (T + K - 1) / K;
    const size_t es = c->precision == LBM_F64 ? 8 : 4;
    const size_t pop_bytes = (size_t)27 * c->stride * c->esize;
    const size_t n = (size_t)d.scells;       // stored cells (adjoint and moment buffers)
    const size_t nd = (size_t)d.cells;       // dense cells (dJ/dg_z)
    // temporaries: checkpoints, a work copy of the populations, per-step moments of one
    // segment, two adjoint buffers, FP64 accumulators
    void *ck = nullptr, *work = nullptr, *mom = nullptr, *lam = nullptr, *accseg = nullptr;
    double *acc = nullptr;
    cudaError_t e = dev_alloc(c, &ck, pop_bytes * (size_t)std::max<int64_t>(nseg - 1, 1));
    if (e == cudaSuccess) e = dev_alloc(c, &work, pop_bytes);
    // two moment buffers when segments are recomputed: the recompute of segment s - 1 fills
    // one while the backward steps of segment s read the other
    const size_t mom_seg = (size_t)K * 9 * n * es;
    if (e == cudaSuccess) e = dev_alloc(c, &mom, mom_seg * (nseg > 1 ? 2 : 1));
    if (e == cudaSuccess) e = dev_alloc(c, &lam, 2 * 27 * n * es);
    if (e == cudaSuccess) e = dev_alloc(c, &accseg, n * es);
    // adjoint kernel: 256 threads over (plane pair, stored position)
    const int64_t nblk = ((int64_t)d.Ps * ((d.nz + lbm::ADJ_ZC - 1) / lbm::ADJ_ZC) + 255) / 256;
    const int64_t nslot = nblk * 8;                  // one slot per warp
    if (e == cudaSuccess) e = dev_alloc(c, (void **)&acc, (nd + 2 * nslot) * sizeof(double));
    auto release = [&]() {
        dev_free(c, ck); dev_free(c, work); dev_free(c, mom); dev_free(c, lam); dev_free(c, acc); dev_free(c, accseg);
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        release();
        return set_err(c, LBM_ENOMEM, "cannot allocate the adjoint buffers (%lld checkpoints of %zu bytes)",
                       (long long)nseg, pop_bytes);
    }
    // the forward pass runs with direct launches of the context's shape, without statistics
    // or checks; they are restored afterwards
    double *stats_save = c->stats;
    const int64_t check_save = c->check_every;
    const int variant_save = c->variant, variant_odd_save = c->variant_odd;
    const int32_t chunk_save = c->graph_chunk;
    c->stats = nullptr;
    c->check_every = 0;
    c->graph_chunk = 0;
    int rc = LBM_OK;
    const int64_t t0 = c->t;
    // forward pass: a checkpoint at the start of every segment but the last, whose steps
    // store their moments at once (its recompute is skipped in the reverse sweep); the
    // moment-storing kernel runs in the shape moments_variant
    for (int64_t sgm = 0; sgm < nseg && rc == LBM_OK; ++sgm) {
        const int64_t ns = std::min<int64_t>(K, T - sgm * K);
        if (sgm < nseg - 1) {
            e = cudaMemcpyAsync((char *)ck + sgm * pop_bytes, c->pops, pop_bytes, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) { rc = cuda_err(c, e, "checkpoint copy"); break; }
            for (int64_t k = 0; k < ns && rc == LBM_OK; ++k) rc = step_direct(c);
        } else {
            c->variant = c->variant_odd = lbm::moments_variant(c->precision);
            for (int64_t k = 0; k < ns && rc == LBM_OK; ++k) {
                StepArgs a = make_args(c, c->t);
                a.moments = (char *)mom + (size_t)(sgm & 1) * mom_seg + (size_t)k * 9 * n * es;
                rc = dispatch(c, [&](auto P) {
                    return lbm::launch_step_moments<decltype(P)::value>((int)(c->t & 1), a, c->stream);
                });
                c->t++;
            }
        }
    }
    const int64_t t_end = c->t;
    int64_t nfl = d.n_fluid;
    lbm::AdjArgs j;
    std::memset(&j, 0, sizeof j);
    j.objective = objective;
    j.kappa = 1.0 / ((double)T * (double)std::max<int64_t>(nfl, 1));
    j.wss = 2.0 / ((double)T * 2.0 * M_PI * d.R * (double)d.nz);
    j.kappa_f = (float)j.kappa;
    j.wss_f = (float)j.wss;
    j.acc = acc;
    j.acc_seg = accseg;
    j.blockacc = acc + nd;
    j.nblocks = (int32_t)nblk;
    if (rc == LBM_OK) {
        e = cudaMemsetAsync(lam, 0, 2 * 27 * n * es, c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, (nd + 2 * nslot) * sizeof(double), c->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(accseg, 0, n * es, c->stream);
        if (e != cudaSuccess) rc = cuda_err(c, e, "adjoint buffer clear");
    }
    // Reverse sweep.  The backward steps of segment s run on the context's stream while the
    // recompute of segment s - 1 (from its checkpoint, storing its moments into the other
    // buffer) runs on a second stream: events order every recompute after the last reader
    // of its buffer (the backward steps of segment s + 1) and every backward segment after
    // its recompute.  Both kernels are latency-bound, so running them side by side keeps
    // more of the GPU busy.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_start = nullptr, ev_rec[2] = {nullptr, nullptr}, ev_bwd[2] = {nullptr, nullptr};
    if (rc == LBM_OK && nseg > 1) {
        e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming);
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cudaEventCreateWithFlags(&ev_rec[b], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_bwd[b], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_start, c->stream);      // checkpoints are written
        if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_start, 0);
        if (e != cudaSuccess) rc = cuda_err(c, e, "adjoint streams");
    }
    auto recompute = [&](int64_t sgm) -> int {
        const int64_t ts = t0 + sgm * K, ns = std::min<int64_t>(K, T - sgm * K);
        cudaError_t ce = cudaMemcpyAsync(work, (char *)ck + sgm * pop_bytes, pop_bytes, cudaMemcpyDeviceToDevice, side);
        if (ce != cudaSuccess) return cuda_err(c, ce, "checkpoint restore");
        for (int64_t k = 0; k < ns; ++k) {
            StepArgs a = make_args(c, ts + k);
            a.pops = work;
            a.moments = (char *)mom + (size_t)(sgm & 1) * mom_seg + (size_t)k * 9 * n * es;
            const int r = dispatch(c, [&](auto P) {
                return lbm::launch_step_moments<decltype(P)::value>((int)((ts + k) & 1), a, side);
            });
            if (r) return r;
        }
        ce = cudaEventRecord(ev_rec[sgm & 1], side);
        return ce == cudaSuccess ? LBM_OK : cuda_err(c, ce, "adjoint event");
    };
    if (rc == LBM_OK && nseg > 1) rc = recompute(nseg - 2);
    for (int64_t sgm = nseg - 1; sgm >= 0 && rc == LBM_OK; --sgm) {
        const int64_t ts = t0 + sgm * K, ns = std::min<int64_t>(K, T - sgm * K);
        if (sgm < nseg - 1) {
            e = cudaStreamWaitEvent(c->stream, ev_rec[sgm & 1], 0);           // its moments are ready
            if (e != cudaSuccess) { rc = cuda_err(c, e, "adjoint event wait"); break; }
        }
        for (int64_t k = ns - 1; k >= 0 && rc == LBM_OK; --k) {
            const int64_t t = ts + k;
            StepArgs a = make_args(c, t);
            j.lam_next = (char *)lam + (size_t)((t + 1) & 1) * 27 * n * es;
            j.lam = (char *)lam + (size_t)(t & 1) * 27 * n * es;
            j.moments = (char *)mom + (size_t)(sgm & 1) * mom_seg + (size_t)k * 9 * n * es;
            rc = dispatch(c, [&](auto P) { return lbm::launch_adjoint<decltype(P)::value>(a, j, c->stream); });
        }
        if (rc == LBM_OK) {
            const StepArgs a = make_args(c, ts);
            rc = dispatch(c, [&](auto P) {
                return lbm::launch_flush_segment<decltype(P)::value>(a, d, j, c->stream);
            });
        }
        if (rc == LBM_OK && sgm >= 2) {
            // the recompute of segment sgm - 2 reuses this segment's moment buffer
            e = cudaEventRecord(ev_bwd[sgm & 1], c->stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_bwd[sgm & 1], 0);
            if (e != cudaSuccess) { rc = cuda_err(c, e, "adjoint event"); break; }
            rc = recompute(sgm - 2);
        }
    }
    if (side) {
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
    }
    for (cudaEvent_t ev : {ev_start, ev_rec[0], ev_rec[1], ev_bwd[0], ev_bwd[1]})
        if (ev) cudaEventDestroy(ev);
    // J and dJ/domega: deterministic sums over cells; dJ/dg_z per cell
    double host[5] = {0, 0, 0, 0, 0};
    if (rc == LBM_OK) {
        double *dout = c->partials + lbm::REDUCE_MAX_BLOCKS * 5;
        rc = dispatch(c, [&](auto P) {
            return lbm::launch_sum_columns<decltype(P)::value>(acc + nd, nslot, 2, c->partials,
                                                               lbm::REDUCE_MAX_BLOCKS, dout, c->stream);
        });
        if (rc == LBM_OK) {
            e = cudaMemcpyAsync(host, dout, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess && dJ_dgz)
                e = cudaMemcpyAsync(dJ_dgz, acc, nd * sizeof(double), cudaMemcpyDefault, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) rc = cuda_err(c, e, "adjoint results");
        }
    }
    c->t = t_end;
    c->stats = stats_save;
    c->check_every = check_save;
    c->variant = variant_save;
    c->variant_odd = variant_odd_save;
    c->graph_chunk = chunk_save;
    cudaStreamSynchronize(c->stream);
    release();
    if (rc) return rc;
    if (J) *J = host[0];
    if (dJ_domega) *dJ_domega = host[1];
    return LBM_OK;
}

int lbm_profile_enable(lbm_ctx *c, int32_t on) {
    if (!c) return LBM_EINVAL;
    c->prof = on != 0;
    return LBM_OK;
}

int lbm_profile_read(lbm_ctx *c, double *ms, int64_t *launches) {
    if (!c) return LBM_EINVAL;
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    double total = 0;
    int64_t n = 0;
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float x = 0;
        LBM_CUDA(c, cudaEventElapsedTime(&x, c->ev[k], c->ev[k + 1]));
        total += x;
        n += c->ev_launches[k / 2];
    }
    if (ms) *ms = total;
    if (launches) *launches = n;
    c->ev_used = 0;
    c->ev_launches.clear();
    return LBM_OK;
}

int lbm_fluid_mask(lbm_ctx *c, uint8_t *mask) {
    if (!c || !mask) return LBM_EINVAL;
    const Member &d = c->hm[c->sel];
    for (int y = 0; y < d.ny; ++y)
        for (int x = 0; x < d.nx; ++x) mask[(size_t)y * d.nx + x] = col_fluid_host(d, x, y) ? 1 : 0;
    return LBM_OK;
}

// ---- checkpoint files ----------------------------------------------------------------
namespace {
struct FileHeader {
    char magic[8];            // "LBMCKPT1"
    int32_t precision, wall, n_members, stats_every;
    int64_t stride, dense_total, t, stats_count, pop_bytes, stats_bytes;
};

bool same_layout(const lbm_ctx *c, const FileHeader &h) {
    return h.precision == c->precision && h.wall == c->wall && h.n_members == (int32_t)c->hm.size() &&
           h.stride == c->stride && h.dense_total == c->dense_total;
}
}  // namespace

int lbm_save(lbm_ctx *c, const char *path) {
    if (!c || !path) return LBM_EINVAL;
    FileHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "LBMCKPT1", 8);
    h.precision = c->precision;
    h.wall = c->wall;
    h.n_members = (int32_t)c->hm.size();
    h.stats_every = c->stats ? c->stats_every : 0;
    h.stride = c->stride;
    h.dense_total = c->dense_total;
    h.t = c->t;
    h.stats_count = c->stats_count;
    h.pop_bytes = (int64_t)27 * c->stride * (int64_t)c->esize;
    h.stats_bytes = c->stats ? (int64_t)sizeof(double) * 4 * c->dense_total : 0;
    std::vector<char> host((size_t)std::max<int64_t>(h.pop_bytes, h.stats_bytes));
    FILE *fp = std::fopen(path, "wb");
    if (!fp) return set_err(c, LBM_EINVAL, "cannot open %s for writing", path);
    bool ok = std::fwrite(&h, sizeof h, 1, fp) == 1;
    cudaError_t e = cudaMemcpyAsync(host.data(), c->pops, (size_t)h.pop_bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    ok = ok && e == cudaSuccess && std::fwrite(host.data(), 1, (size_t)h.pop_bytes, fp) == (size_t)h.pop_bytes;
    if (ok && h.stats_bytes) {
        e = cudaMemcpyAsync(host.data(), c->stats, (size_t)h.stats_bytes, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        ok = e == cudaSuccess && std::fwrite(host.data(), 1, (size_t)h.stats_bytes, fp) == (size_t)h.stats_bytes;
    }
    ok = (std::fclose(fp) == 0) && ok;
    if (e != cudaSuccess) return cuda_err(c, e, "checkpoint download");
    if (!ok) return set_err(c, LBM_EINVAL, "writing %s failed", path);
    return LBM_OK;
}

int lbm_load(lbm_ctx *c, const char *path) {
    if (!c || !path) return LBM_EINVAL;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return set_err(c, LBM_EINVAL, "cannot open %s", path);
    FileHeader h;
    bool ok = std::fread(&h, sizeof h, 1, fp) == 1 && std::memcmp(h.magic, "LBMCKPT1", 8) == 0;
    // the header must describe exactly this context's buffers before anything is read
    // into them: the population bytes of this layout, and either no statistics or
    // 4 FP64 sums per dense cell with a sampling interval >= 1 and a count >= 0
    const int64_t pop_need = (int64_t)27 * c->stride * (int64_t)c->esize;
    const int64_t stats_need = (int64_t)sizeof(double) * 4 * c->dense_total;
    if (!ok || !same_layout(c, h) || h.pop_bytes != pop_need ||
        (h.stats_bytes != 0 && (h.stats_bytes != stats_need || h.stats_every < 1 || h.stats_count < 0)) ||
        h.t < 0) {
        std::fclose(fp);
        return set_err(c, LBM_EINVAL, "%s is not a checkpoint of a context with this layout", path);
    }
    // read the whole file into host memory first; the context changes only once all
    // of it has been read
    std::vector<char> pops((size_t)h.pop_bytes), stats((size_t)h.stats_bytes);
    ok = std::fread(pops.data(), 1, pops.size(), fp) == pops.size() &&
         std::fread(stats.data(), 1, stats.size(), fp) == stats.size();
    std::fclose(fp);
    if (!ok) return set_err(c, LBM_EINVAL, "reading %s failed (file truncated)", path);
    if (h.stats_bytes && !c->stats) {
        int rc = lbm_stats_enable(c, h.stats_every);
        if (rc) return rc;
    }
    cudaError_t e = cudaMemcpyAsync(c->pops, pops.data(), pops.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && h.stats_bytes)
        e = cudaMemcpyAsync(c->stats, stats.data(), stats.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_err(c, e, "checkpoint upload");
    if (h.stats_bytes) {
        c->stats_every = h.stats_every;
        c->stats_count = h.stats_count;
    }
    c->t = h.t;
    for (size_t m = 0; m < c->hm.size(); ++m) c->mass0_valid[m] = false;
    return LBM_OK;
}

}  // extern "C"
