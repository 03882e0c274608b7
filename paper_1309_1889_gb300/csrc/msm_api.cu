// msm_api.cu -- the C ABI of libmsm_gb300.so (declared in include/msm.h):
// handle and scratch management, geometry and table set-up, and the
// orchestration of one MSM evaluation (Sec. 3, worked example steps 1-9),
// of velocity Verlet (Sec. 2) and of parareal (Sec. 4).  Every evaluation
// and every MD step serves a batch of independent systems with one launch
// per stage (a single system is the batch of one); MD steps after the first
// replay a captured CUDA graph.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <vector>

#include "kernels.cuh"

using namespace msm;

// ------------------------------------------------------------------ errors

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_alloc_gen{0};     // bumped by every device (re)allocation

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

int fail_cuda(cudaError_t e, const char *what, const char *file, int line)
{
    snprintf(g_err, sizeof g_err, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MSM_ENOMEM : MSM_ECUDA;
}

int fail_msg(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return code;
}

#define TRY(expr)                     \
    do {                              \
        int rc__ = (expr);            \
        if (rc__ != MSM_OK) return rc__; \
    } while (0)

static const char *status_text(int s)
{
    switch (s) {
    case MSM_EINVAL: return "non-finite coordinate";
    case MSM_ERANGE: return "an atom lies outside the box";
    case MSM_ENOCONV: return "SHAKE/RATTLE did not converge";
    case MSM_ETIMEOUT: return "a device-side wait ran out";
    default: return "device error";
    }
}

// ----------------------------------------------------------------- buffers

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    template <typename X> X *as() const { return static_cast<X *>(p); }
};

// Device bytes the library holds (every handle's buffers) and the caller's budget for them
static std::atomic<long long> g_held_bytes{0}, g_budget_bytes{0};

static int ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return MSM_OK;
    if (b.p) { cudaFree(b.p); g_held_bytes.fetch_sub((long long)b.cap); }
    b.p = nullptr;
    b.cap = 0;
    g_alloc_gen.fetch_add(1);
    const long long budget = g_budget_bytes.load();
    if (budget > 0 && g_held_bytes.load() + (long long)bytes > budget)
        return fail_msg(MSM_ENOMEM, "device memory budget of %lld bytes exceeded (%lld held, %zu more needed)",
                        budget, g_held_bytes.load(), bytes);
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail_msg(MSM_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    g_held_bytes.fetch_add((long long)bytes);
    return MSM_OK;
}

static void release(DevBuf &b)
{
    if (b.p) { cudaFree(b.p); g_held_bytes.fetch_sub((long long)b.cap); }
    b.p = nullptr;
    b.cap = 0;
}

extern "C" int64_t msm_set_device_budget(int64_t bytes)
{
    g_budget_bytes.store(bytes > 0 ? (long long)bytes : 0);
    return (int64_t)g_held_bytes.load();
}

// Device memory of the current device, or managed memory: used in place.
// Anything else is treated as host memory and staged (see foreign_device).
static bool on_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.device == dev;
}

// A device allocation made on a GPU other than the current one.  The kernels
// run on the current device and would dereference it there (an illegal
// address without peer access), and staging it as host memory is wrong too,
// so every entry point rejects such arrays with MSM_EINVAL before any launch.
static bool foreign_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return true; }
    return at.device != dev;
}

static int check_arrays(std::initializer_list<const void *> ptrs)
{
    for (const void *p : ptrs)
        if (foreign_device(p))
            return fail_msg(MSM_EINVAL, "an array lives on another GPU than the current device");
    return MSM_OK;
}

// ------------------------------------------------------------------ handle

// Stages timed by the profiler (CUDA events around each stage's launches).
enum Stage { ST_BIN, ST_SHORT, ST_ANTERP, ST_RESTRICT, ST_STENCIL, ST_TOP, ST_PROLONG, ST_INTERP, ST_SUMS,
             ST_VV1, ST_VV2, ST_LIST, ST_LJ, N_STAGES };
static const char *kStageNames[N_STAGES] = {"bin_sort",      "short_range", "anterpolation",
                                            "restriction",   "lattice_cutoff", "top_level",
                                            "prolongation",  "interpolation", "exclusions_sums",
                                            "vv_first_shake", "vv_second_rattle", "verlet_list_maintenance",
                                            "lennard_jones"};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    std::vector<int3> marks;        // (stage, begin event, end event)
    double ms[N_STAGES] = {0};
    long long cnt[N_STAGES] = {0};
};

// One system of a batch as the host sees it.
struct SysIn {
    int64_t n, n_mol;
    double box[6];
};

// What a captured md step depends on: a replay is valid only while all of it
// is unchanged (device buffers are identified by the allocation generation).
struct GraphKey {
    const void *x, *v, *f, *q, *m, *lj, *uk;
    long long uk_stride, geom_gen, alloc_gen;
    double dt;
    int B, list_on, mts;
};

// Brick shape chosen by timing, per system geometry (atoms, cells per axis).
struct Tuned {
    long long n;
    int nc[3];
    int bd[3];
    int lj_bd[3];          // bricks of the LJ pass (water model; 0 = not tuned)
    int gcw, lgcw;         // column widths of the i groups, all atoms and LJ sites (0 = not tuned)
};

struct msm_handle {
    msm_params p;
    Profiler prof;
    int precision;
    // batch geometry: B systems, concatenated atoms / cells / grids
    bool have_geom = false;
    int B = 0;
    std::vector<SysIn> sys_key;
    std::vector<SysDesc> hsd;
    std::vector<int> h_blk;
    std::vector<CUtensorMap> st_maps;                   // TMA descriptors of the lattice-cutoff planes
    long long geom_gen = 0;
    int N = 0, M = 0, G = 0, UT = 0, TT = 0, PB = 0, stiles = 0;
    int max_n = 0, max_mol = 0, max_units = 0, max_bricks = 0, max_atiles = 0, max_top = 0, max_lj_bricks = 0;
    int max_lev[MSM_MAX_LEVELS] = {0};
    DevBuf sd_buf, blk_buf;
    // system 0 of the batch (inspection and Verlet lists)
    double box[6] = {0, 0, 0, 0, 0, 0};
    CellGeom cg;
    GridGeom gg;
    double inv_h = 0;
    int bd[3] = {4, 2, 2}, nb[3] = {0, 0, 0}, nbricks = 0;
    int64_t last_n = 0;
    // brick autotuner
    std::vector<Tuned> tuned;
    bool tune_pending = false;
    // tables
    bool stencil_ready = false;
    StencilGeom sg;
    // scratch
    DevBuf key, count, start, perm, bsum, rel, frac, apos, afrac, akey, aflag, aw, sr, lj;
    DevBuf lj_count, lj_start, lj_apos, lj_flag, lj_perm;      // LJ-site cell list (water completion)
    DevBuf qgrid, ucut, ugrid, utop, ttop, wst_d, wst_t, rows;
    DevBuf eatom, vatom, kin, partials, sums, kin_s, status, ctr;
    DevBuf in_pos, in_q, in_lj, out_f, out_p;          // staging of host arrays
    DevBuf md_f, md_xo, md_x, md_v, md_q, md_m, md_lj, md_uk, md_im;
    DevBuf md_fs, eslow;                                // multiple time stepping: slow forces and energies
    int *h_status = nullptr;
    double *h_scal = nullptr;
    double *h_e = nullptr;                              // pinned, per-system energies
    int h_e_cap = 0;
    // CUDA graph of one md step
    cudaStream_t cap_st = nullptr;
    cudaStream_t grid_st = nullptr;                     // high-priority stream of the grid chain
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    long long g_kernels = 0;                            // kernels per replayed step
    // Verlet lists (md_run with list_skin > 0, single systems)
    bool list_on = false;
    // i groups of the pair passes (off with MSM_FLAG_BRICKS); lgp_*: the LJ-site pass
    bool gp_on = false;
    int gp_cols = 0, gp_max_cols = 0, gp_max_groups = 0, lgp_cols = 0, lgp_max_cols = 0, lgp_max_groups = 0;
    int gp_max_nz = 0;                                  // cell layers of the largest system
    DevBuf gp_cnt, gp_col, gp_bsum, gp_slot, lgp_cnt, lgp_col, lgp_bsum, lgp_slot;
    // cluster pairs (MSM_FLAG_CLUSTER_PAIRS)
    bool cp_on = false;
    int cp_cols = 0, cp_max_cols = 0, cp_max_icl = 0;
    DevBuf cp_coln, cp_colcl, cp_bsum, cp_zc, cp_pos, cp_mol, cp_slot, cp_box;
    DevBuf vl_perm, vl_start, vl_xref, vl_pos, vl_rtab, vl_rtn, vl_cnt, vl_cntlj, vl_nbr, vl_nbr_lj, vl_ctl;
    int vl_cap = 0, vl_cap_lj = 0, vl_nbricks = 0;
    int64_t vl_key_n = -1, vl_key_nmol = -1;
    double vl_key_box[6] = {0, 0, 0, 0, 0, 0};
    const void *vl_key_lj = nullptr;
    int *h_ctl = nullptr;
    int64_t vl_builds = 0, vl_overflows = 0, vl_seen[3] = {0, 0, 0};
};

static int prof_event(msm_handle *h, cudaStream_t st, int *idx)
{
    Profiler &P = h->prof;
    if (P.used == P.ev.size()) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        P.ev.push_back(e);
    }
    *idx = (int)P.used++;
    CUDA_TRY(cudaEventRecord(P.ev[*idx], st));
    return MSM_OK;
}

// Scope guard: records a begin event now and an end event when it leaves scope.
struct ProfScope {
    msm_handle *h;
    cudaStream_t st;
    int stage, b = -1;
    ProfScope(msm_handle *h_, int stage_, cudaStream_t st_) : h(h_), st(st_), stage(stage_)
    {
        if (h->prof.on && prof_event(h, st, &b) != MSM_OK) b = -1;
    }
    ~ProfScope()
    {
        int e;
        if (b >= 0 && prof_event(h, st, &e) == MSM_OK) h->prof.marks.push_back(make_int3(stage, b, e));
    }
};
#define PROF(stage) ProfScope prof_scope__(h, stage, st)

// After a stream synchronisation: fold the recorded event pairs into the totals.
static void prof_resolve(msm_handle *h)
{
    Profiler &P = h->prof;
    for (const int3 &m : P.marks) {
        float t = 0;
        if (cudaEventElapsedTime(&t, P.ev[m.y], P.ev[m.z]) == cudaSuccess) {
            P.ms[m.x] += t;
            P.cnt[m.x] += 1;
        } else {
            cudaGetLastError();
        }
    }
    P.marks.clear();
    P.used = 0;
}

extern "C" void msm_default_params(msm_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof *p);
    p->a = 1.2;
    p->h = 0.25;
    p->n_levels = 3;
    p->precision = MSM_FP32;
    p->coulomb_k = 138.935458;
    p->gamma_kind = 0;
    p->basis_kind = 0;
    p->model = MSM_MODEL_CHARGES;
    p->flags = MSM_FLAG_GRAPHS | MSM_FLAG_AUTOTUNE;
    p->lj_sigma = 0.315061;
    p->lj_epsilon = 0.6364;
    p->d_oh = 0.09572;
    p->d_hh = 2.0 * 0.09572 * sin(104.52 * M_PI / 360.0);
    p->wall_k = 0.0;
    p->wall_width = 0.0;
    p->list_skin = 0.0;
    p->method = MSM_METHOD_MSM;
    p->mts_steps = 0;
    p->wolf_alpha = 0.0;
}

static bool has_grids(const msm_params &p) { return p.method == MSM_METHOD_MSM; }

static int check_params(const msm_params *p)
{
    if (!p) return fail_msg(MSM_EINVAL, "params is NULL");
    if (!(p->a > 0) || !(p->h > 0) || !std::isfinite(p->a) || !std::isfinite(p->h))
        return fail_msg(MSM_EINVAL, "a and h must be positive and finite");
    if (p->n_levels < 1 || p->n_levels > MSM_MAX_LEVELS)
        return fail_msg(MSM_EINVAL, "n_levels must be in 1..%d", MSM_MAX_LEVELS);
    if (p->precision != MSM_FP32 && p->precision != MSM_FP64) return fail_msg(MSM_EINVAL, "unknown precision");
    if (p->gamma_kind != 0 || p->basis_kind != 0) return fail_msg(MSM_EINVAL, "only gamma_kind 0 and basis_kind 0 exist");
    if (p->model != MSM_MODEL_CHARGES && p->model != MSM_MODEL_WATER) return fail_msg(MSM_EINVAL, "unknown model");
    if (p->flags & ~(MSM_FLAG_GRAPHS | MSM_FLAG_AUTOTUNE | MSM_FLAG_SCALAR_PAIRS | MSM_FLAG_CLUSTER_PAIRS |
                     MSM_FLAG_BRICKS))
        return fail_msg(MSM_EINVAL, "unknown flags");
    if (!(p->wall_k >= 0) || !(p->wall_width >= 0)) return fail_msg(MSM_EINVAL, "wall_k and wall_width must be >= 0");
    if (!(p->list_skin >= 0) || !(p->list_skin < p->a)) return fail_msg(MSM_EINVAL, "list_skin must be in [0, a)");
    if (p->method != MSM_METHOD_MSM && p->method != MSM_METHOD_CUTOFF && p->method != MSM_METHOD_WOLF)
        return fail_msg(MSM_EINVAL, "unknown method");
    if (!(p->wolf_alpha >= 0) || !std::isfinite(p->wolf_alpha)) return fail_msg(MSM_EINVAL, "wolf_alpha must be >= 0");
    if (p->method == MSM_METHOD_WOLF && p->list_skin > 0)
        return fail_msg(MSM_EINVAL, "Verlet lists serve the MSM and the simple cutoff only");
    if (p->mts_steps < 0) return fail_msg(MSM_EINVAL, "mts_steps must be >= 0");
    if (p->mts_steps > 1 && p->method != MSM_METHOD_MSM)
        return fail_msg(MSM_EINVAL, "multiple time stepping needs the MSM (the cutoff methods have no slow part)");
    if (p->method != MSM_METHOD_MSM) return MSM_OK;          // no grids: n_levels is not used
    int rad = 0;
    while ((double)(rad + 1) * p->h < 2.0 * p->a) rad++;
    if (rad > 12 && p->n_levels > 1)                       // one level has no lattice cutoff
        return fail_msg(MSM_EINVAL, "2a/h = %.3g is too large (lattice-cutoff radius %d > 12)", 2 * p->a / p->h, rad);
    return MSM_OK;
}

extern "C" int msm_create(const msm_params *p, msm_handle **out)
{
    if (!out) return fail_msg(MSM_EINVAL, "out is NULL");
    *out = nullptr;
    TRY(check_params(p));
    msm_handle *h = new msm_handle();
    h->p = *p;
    if (!(h->p.coulomb_k > 0)) h->p.coulomb_k = 138.935458;
    h->precision = p->precision;
    memset(&h->gkey, 0, sizeof h->gkey);
    cudaError_t e = cudaMallocHost(&h->h_status, sizeof(int) * 4);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_scal, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMallocHost(&h->h_ctl, sizeof(int) * 8);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail_msg(MSM_ECUDA, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    }
    *out = h;
    g_err[0] = 0;
    return MSM_OK;
}

extern "C" void msm_destroy(msm_handle *h)
{
    if (!h) return;
    DevBuf *all[] = {&h->key, &h->count, &h->start, &h->perm, &h->bsum, &h->rel, &h->frac, &h->apos, &h->afrac,
                     &h->aw, &h->akey, &h->aflag, &h->sr, &h->lj, &h->lj_count, &h->lj_start, &h->lj_apos, &h->lj_flag,
                     &h->lj_perm, &h->qgrid, &h->ucut, &h->ugrid, &h->utop, &h->ttop,
                     &h->wst_d, &h->wst_t, &h->rows, &h->eatom, &h->vatom, &h->kin, &h->partials, &h->sums,
                     &h->kin_s, &h->status, &h->ctr, &h->sd_buf, &h->blk_buf,
                     &h->in_pos, &h->in_q, &h->in_lj, &h->out_f, &h->out_p, &h->md_f, &h->md_xo,
                     &h->md_x, &h->md_v, &h->md_q, &h->md_m, &h->md_lj, &h->md_uk, &h->md_im,
                     &h->md_fs, &h->eslow,
                     &h->vl_perm, &h->vl_start, &h->vl_xref, &h->vl_pos, &h->vl_rtab, &h->vl_rtn,
                     &h->vl_cnt, &h->vl_cntlj, &h->vl_nbr, &h->vl_nbr_lj, &h->vl_ctl,
                     &h->cp_coln, &h->cp_colcl, &h->cp_bsum, &h->cp_zc, &h->cp_pos, &h->cp_mol, &h->cp_slot,
                     &h->cp_box, &h->gp_cnt, &h->gp_col, &h->gp_bsum, &h->gp_slot, &h->lgp_cnt, &h->lgp_col,
                     &h->lgp_bsum, &h->lgp_slot};
    for (DevBuf *b : all) release(*b);
    for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_st) cudaStreamDestroy(h->cap_st);
    if (h->grid_st) cudaStreamDestroy(h->grid_st);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    if (h->h_e) cudaFreeHost(h->h_e);
    delete h;
}

static int64_t floordiv64(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

// Pinned host array of per-system energies, at least B entries.
static int ensure_host_e(msm_handle *h, int B)
{
    if (h->h_e_cap >= B) return MSM_OK;
    if (h->h_e) cudaFreeHost(h->h_e);
    h->h_e = nullptr;
    h->h_e_cap = 0;
    CUDA_TRY(cudaMallocHost(&h->h_e, sizeof(double) * (size_t)std::max(B, 8)));
    h->h_e_cap = std::max(B, 8);
    return MSM_OK;
}

// Brick shape for the short-range kernel: about 24 atoms per warp at the
// system's mean density (one i atom per lane), unless the autotuner timed
// this geometry.  The shape changes only the speed, never the results: each
// i atom sums its j's in ascending slot order whatever the brick.
static const int kNumShapes = 12;
static const int kBrickShapes[kNumShapes][3] = {{1, 1, 1}, {2, 1, 1}, {2, 2, 1}, {2, 2, 2}, {3, 2, 2}, {4, 2, 2},
                                                {3, 3, 2}, {5, 2, 2}, {4, 3, 2}, {4, 4, 2}, {4, 4, 3}, {4, 4, 4}};

// The largest shape (by volume) that holds at most ~28 atoms at the mean density
// (at most one i atom per lane of a warp).
static int brick_heuristic(int64_t n, const CellGeom &g, double target = 28.0)
{
    const double per_cell = (double)n / (double)g.ncells;
    int pick = 0;
    for (int s = 0; s < kNumShapes; s++) {
        const int vol = kBrickShapes[s][0] * kBrickShapes[s][1] * kBrickShapes[s][2];
        if (per_cell * vol <= target) pick = s;
    }
    return pick;
}

static void set_lj_bricks(SysDesc &D, const int bd[3])
{
    for (int k = 0; k < 3; k++) {
        D.lj_bd[k] = bd[k];
        D.lj_nb[k] = (D.g.nc[k] + bd[k] - 1) / bd[k];
    }
    D.lj_nbricks = D.lj_nb[0] * D.lj_nb[1] * D.lj_nb[2];
}

static void set_bricks(SysDesc &D, const int bd[3])
{
    for (int d = 0; d < 3; d++) {
        D.bd[d] = bd[d];
        D.nb[d] = (D.g.nc[d] + bd[d] - 1) / bd[d];
    }
    D.nbricks = D.nb[0] * D.nb[1] * D.nb[2];
}

// Column width of the i groups: columns of cw x cw cells, cw^3 cells holding ~32
// atoms at the mean density.
static int group_width(double per_cell)
{
    const int cw = (int)lround(cbrt(32.0 / std::max(per_cell, 1e-3)));
    return std::min(std::max(cw, 1), 8);
}

// Column layout of the pair passes' i groups from each system's column widths
// (SysDesc::gp_cw, lgp_cw): columns per axis, global column offsets, the bounds
// on the group counts, and (groups on) the buffers.
static int layout_groups(msm_handle *h, std::vector<SysDesc> &d)
{
    int64_t GC = 0, GK = 0, GI = 0, GMAX = 0, LC = 0, LK = 0, LI = 0, LMAX = 0;
    int mnz = 0;
    for (SysDesc &D : d) {
        const int64_t n = D.n, n_lj = (int64_t)D.n_mol + (D.n - 3 * (int64_t)D.n_mol);
        D.gp_nc[0] = (D.g.nc[0] + D.gp_cw - 1) / D.gp_cw;
        D.gp_nc[1] = (D.g.nc[1] + D.gp_cw - 1) / D.gp_cw;
        const int64_t ng = (int64_t)D.gp_nc[0] * D.gp_nc[1];
        D.gp_col_off = (int)GC;
        GC += ng;
        GK += n / 32 + ng;                                 // groups: at most n/32 + 1 per column
        GI = std::max(GI, n / 32 + ng);
        GMAX = std::max(GMAX, ng);
        D.lgp_nc[0] = (D.g.nc[0] + D.lgp_cw - 1) / D.lgp_cw;
        D.lgp_nc[1] = (D.g.nc[1] + D.lgp_cw - 1) / D.lgp_cw;
        const int64_t nl = (int64_t)D.lgp_nc[0] * D.lgp_nc[1];
        D.lgp_col_off = (int)LC;
        LC += nl;
        LK += n_lj / 32 + nl;
        LI = std::max(LI, n_lj / 32 + nl);
        LMAX = std::max(LMAX, nl);
        mnz = std::max(mnz, D.g.nc[2]);
    }
    const int64_t lim = ((int64_t)1 << 31) - 1;
    if (GC >= lim || LC >= lim || 32 * (GK + 1) >= lim || 32 * (LK + 1) >= lim)
        return fail_msg(MSM_EINVAL, "batch too large for 32-bit group offsets");
    if (h->gp_on) {
        TRY(ensure(h->gp_cnt, sizeof(int) * (size_t)(GC + 1)));
        TRY(ensure(h->gp_col, sizeof(int) * (size_t)(GC + 1)));
        TRY(ensure(h->gp_bsum, sizeof(int) * (size_t)scan_scratch_ints((int)GC)));
        TRY(ensure(h->gp_slot, sizeof(int) * 32 * (size_t)(GK + 1)));
        if (h->p.model == MSM_MODEL_WATER) {
            TRY(ensure(h->lgp_cnt, sizeof(int) * (size_t)(LC + 1)));
            TRY(ensure(h->lgp_col, sizeof(int) * (size_t)(LC + 1)));
            TRY(ensure(h->lgp_bsum, sizeof(int) * (size_t)scan_scratch_ints((int)LC)));
            TRY(ensure(h->lgp_slot, sizeof(int) * 32 * (size_t)(LK + 1)));
        }
    }
    h->gp_cols = (int)GC; h->gp_max_cols = (int)GMAX; h->gp_max_groups = (int)GI;
    h->lgp_cols = (int)LC; h->lgp_max_cols = (int)LMAX; h->lgp_max_groups = (int)LI;
    h->gp_max_nz = mnz;
    return MSM_OK;
}

static const Tuned *find_tuned(const msm_handle *h, int64_t n, const CellGeom &g)
{
    for (const Tuned &t : h->tuned)
        if (t.n == n && t.nc[0] == g.nc[0] && t.nc[1] == g.nc[1] && t.nc[2] == g.nc[2]) return &t;
    return nullptr;
}

// Geometry of a batch of systems: cells, grid levels and bricks per system,
// their offsets in the concatenated buffers, the top-level tables (one per
// distinct top shape) and the lattice-cutoff tile offsets of every (system,
// level).  Grid extents per level (open boundaries): level 0 spans
// [-1, floor(L/h)+2]; level k+1 spans [ceil((lo-3)/2), floor((hi+3)/2)], every
// point with a non-zero restriction weight from level k.  Nothing is redone
// while the systems' atom counts and boxes stay the same.
static int ensure_atoms(msm_handle *h, int64_t n);

static int set_batch(msm_handle *h, int B, const SysIn *sys, cudaStream_t st)
{
    if (B < 1) return fail_msg(MSM_EINVAL, "a batch needs at least one system");
    for (int s = 0; s < B; s++) {
        const SysIn &S = sys[s];
        for (int d = 0; d < 6; d++)
            if (!std::isfinite(S.box[d])) return fail_msg(MSM_EINVAL, "box of system %d has a non-finite entry", s);
        for (int d = 0; d < 3; d++)
            if (!(S.box[3 + d] > 0)) return fail_msg(MSM_EINVAL, "box lengths must be positive (system %d)", s);
        if (S.n < 0 || S.n > ((int64_t)1 << 30)) return fail_msg(MSM_EINVAL, "atom count %lld out of range", (long long)S.n);
        if (S.n_mol < 0 || 3 * S.n_mol > S.n) return fail_msg(MSM_EINVAL, "n_mol inconsistent with n (system %d)", s);
    }
    bool same = h->have_geom && B == h->B && !h->tune_pending;
    for (int s = 0; same && s < B; s++)
        same = sys[s].n == h->sys_key[s].n && sys[s].n_mol == h->sys_key[s].n_mol &&
               memcmp(sys[s].box, h->sys_key[s].box, sizeof sys[s].box) == 0;
    if (same) return MSM_OK;
    // until this rebuild completes the handle describes no batch: a failure below (an
    // allocation beyond the budget, say) must not leave a later call reusing buffers
    // that were freed on the way
    h->have_geom = false;

    const double hh = h->p.h;
    const bool grids = has_grids(h->p);
    const int l = grids ? h->p.n_levels : 1;              // the cutoff methods keep level 0's geometry only
    std::vector<SysDesc> d((size_t)B);
    std::vector<std::array<int, 4>> tops;          // (nx, ny, nz, table offset)
    int64_t N = 0, M = 0, G = 0, UT = 0, TT = 0, PB = 0, ST = 0;
    int64_t CC = 0, CZ = 0, CK = 0, CI = 0, CMAX = 0;    // cluster pairs: columns, layer tables, clusters of 4
    bool pending = false;
    h->h_blk.clear();
    for (int s = 0; s < B; s++) {
        SysDesc &D = d[(size_t)s];
        memset(&D, 0, sizeof D);
        const SysIn &S = sys[s];
        int64_t ncells = 1;
        for (int k = 0; k < 3; k++) {
            D.g.origin[k] = S.box[k];
            const double nc = floor(S.box[3 + k] / hh) + 1.0;
            if (nc > 4.0e6) return fail_msg(MSM_EINVAL, "box too large for h");
            D.g.nc[k] = (int)nc;
            ncells *= D.g.nc[k];
            D.box_lo[k] = S.box[k];
            D.box_hi[k] = S.box[k] + S.box[3 + k];
        }
        if (ncells > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "too many cells (%lld)", (long long)ncells);
        D.g.h = hh;
        D.g.ncells = (int)ncells;
        D.inv_h = 1.0 / hh;
        for (int k = 0; k < 3; k++) {
            D.wall_lo[k] = (int)floor(h->p.wall_width * D.inv_h) + 2;
            D.wall_hi[k] = (int)floor((S.box[3 + k] - h->p.wall_width) * D.inv_h) - 2;
        }
        D.gg.levels = l;
        // Level ranges: level 0 spans [-1, floor(L/h) + 2], level k+1 [ceil((lo-3)/2),
        // floor((hi+3)/2)] of level k.  Each level's x range is then extended to a
        // multiple of 4 points (hi_x grows by up to 3, and the next level's range
        // derives from the extended one): rows start on 16-byte boundaries, as the
        // TMA copies of the lattice cutoff need.  The added points
        // carry zero charge at every level (a point gets charge only from points
        // within its restriction taps, all inside the unextended range), and no
        // point of the unextended range reads a potential outside it, so the
        // extension changes no result.
        int64_t lo[3], hi[3], hi_log = 0, tot = 0;
        for (int k = 0; k < 3; k++) { lo[k] = -1; hi[k] = (int64_t)floor(S.box[3 + k] / hh) + 2; }
        hi_log = hi[0];
        for (int k = 0; k < l; k++) {
            if (k > 0) {
                for (int e = 0; e < 3; e++) { lo[e] = -floordiv64(-(lo[e] - 3), 2); hi[e] = floordiv64(hi[e] + 3, 2); }
                hi_log = floordiv64(hi_log + 3, 2);
            }
            const int64_t nx_log = hi_log - lo[0] + 1, nx_ext = hi[0] - lo[0] + 1;
            hi[0] = lo[0] + ((nx_ext + 3) / 4) * 4 - 1;
            int64_t sz = 1;
            for (int e = 0; e < 3; e++) {
                D.gg.L[k].lo[e] = (int)lo[e];
                D.gg.L[k].n[e] = (int)(hi[e] - lo[e] + 1);
                sz *= D.gg.L[k].n[e];
            }
            D.gg.L[k].nx_log = (int)nx_log;
            D.gg.L[k].off = (int)tot;
            tot += sz;
        }
        if (tot > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "grids too large");
        D.gg.total = (int)tot;
        D.atom_off = (int)N;
        D.n = (int)S.n;
        D.n_mol = (int)S.n_mol;
        N += S.n;
        D.cell_off = (int)M;
        M += ncells;
        D.cp_nc[0] = (D.g.nc[0] + 1) / 2;
        D.cp_nc[1] = (D.g.nc[1] + 1) / 2;
        {
            const int64_t nco = (int64_t)D.cp_nc[0] * D.cp_nc[1], n = (int64_t)S.n;
            D.col_off = (int)CC;
            D.zc_off = (int)CZ;
            CC += nco;
            CZ += nco * (D.g.nc[2] + 1);
            CK += n / 4 + 2 * nco;                         // clusters of 4: at most n/4 + 2 per column
            CI = std::max(CI, n / 8 + nco);                 // i clusters: at most n/8 + 1 per column
            CMAX = std::max(CMAX, nco);
        }
        const Tuned *t = (h->p.flags & MSM_FLAG_AUTOTUNE) ? find_tuned(h, S.n, D.g) : nullptr;
        {
            const int64_t n_lj = (int64_t)(S.n_mol + (S.n - 3 * S.n_mol));
            D.gp_cw = (t && t->gcw) ? t->gcw : group_width((double)S.n / (double)ncells);
            D.lgp_cw = (t && t->lgcw) ? t->lgcw : group_width((double)n_lj / (double)ncells);
        }
        if (t) set_bricks(D, t->bd);
        else {
            set_bricks(D, kBrickShapes[brick_heuristic(S.n, D.g)]);
            if ((h->p.flags & MSM_FLAG_AUTOTUNE) && S.n > 0) pending = true;
        }
        if (h->p.model == MSM_MODEL_WATER) {
            // LJ pass: the O sites and single sites of the water completion
            const int n_lj = (int)(S.n_mol + (S.n - 3 * S.n_mol));
            set_lj_bricks(D, (t && t->lj_bd[0]) ? t->lj_bd : kBrickShapes[brick_heuristic(n_lj, D.g)]);
        }
        D.part_off = (int)PB;
        PB += sum_blocks((int)S.n);
        if (!grids) continue;                              // no grid buffers, tables or tiles
        D.grid_off = (int)G;
        G += tot;
        const LevelGeom &Lt = D.gg.L[l - 1];
        D.top_off = (int)UT;
        UT += (int64_t)Lt.n[0] * Lt.n[1] * Lt.n[2];
        int found = -1;
        for (size_t k = 0; k < tops.size(); k++)
            if (tops[k][0] == Lt.n[0] && tops[k][1] == Lt.n[1] && tops[k][2] == Lt.n[2]) found = (int)k;
        if (found < 0) {
            tops.push_back({Lt.n[0], Lt.n[1], Lt.n[2], (int)TT});
            TT += (int64_t)(2 * Lt.n[0] - 1) * (2 * Lt.n[1] - 1) * (2 * Lt.n[2] - 1);
            found = (int)tops.size() - 1;
        }
        D.ttab_off = tops[(size_t)found][3];
        for (int k = 0; k + 1 < l; k++) {
            h->h_blk.push_back((int)ST);
            ST += stencil_tile_count(D.gg.L[k]);
        }
    }
    h->h_blk.push_back((int)ST);
    const int64_t lim = ((int64_t)1 << 31) - 1;
    if (N > ((int64_t)1 << 30) || M >= lim || G >= lim || UT >= lim || TT >= lim || ST >= lim || CZ >= lim ||
        4 * CK >= lim)
        return fail_msg(MSM_EINVAL, "batch too large for 32-bit offsets");

    const size_t ts = h->precision == MSM_FP32 ? sizeof(float) : sizeof(double);
    TRY(ensure(h->count, sizeof(int) * (size_t)(M + 1)));
    TRY(ensure(h->start, sizeof(int) * (size_t)(M + 1)));
    if (h->p.model == MSM_MODEL_WATER) {
        TRY(ensure(h->lj_count, sizeof(int) * (size_t)(M + 1)));
        TRY(ensure(h->lj_start, sizeof(int) * (size_t)(M + 1)));
    }
    TRY(ensure(h->bsum, sizeof(int) * (size_t)scan_scratch_ints((int)M)));
    h->gp_on = !(h->p.flags & MSM_FLAG_BRICKS);
    TRY(layout_groups(h, d));
    h->cp_on = (h->p.flags & MSM_FLAG_CLUSTER_PAIRS) && h->precision == MSM_FP32 &&
               h->p.method != MSM_METHOD_WOLF && !(h->p.flags & MSM_FLAG_SCALAR_PAIRS);
    if (h->cp_on) {
        TRY(ensure(h->cp_coln, sizeof(int) * (size_t)(CC + 1)));
        TRY(ensure(h->cp_colcl, sizeof(int) * (size_t)(CC + 1)));
        TRY(ensure(h->cp_bsum, sizeof(int) * (size_t)scan_scratch_ints((int)CC)));
        TRY(ensure(h->cp_zc, sizeof(int) * (size_t)CZ));
        TRY(ensure(h->cp_pos, sizeof(float) * 16 * (size_t)CK));
        TRY(ensure(h->cp_mol, sizeof(int) * 4 * (size_t)CK));
        TRY(ensure(h->cp_slot, sizeof(int) * 4 * (size_t)CK));
        TRY(ensure(h->cp_box, sizeof(float) * 8 * (size_t)CK));
    }
    TRY(ensure(h->qgrid, ts * (size_t)G));
    TRY(ensure(h->ucut, ts * (size_t)G));
    TRY(ensure(h->ugrid, ts * (size_t)G));
    TRY(ensure(h->utop, sizeof(double) * (size_t)UT));
    TRY(ensure(h->ttop, sizeof(double) * (size_t)TT));
    TRY(ensure(h->partials, sizeof(double) * 4 * (size_t)PB));
    TRY(ensure(h->sums, sizeof(double) * 4 * (size_t)B));
    TRY(ensure(h->kin_s, sizeof(double) * (size_t)B));
    TRY(ensure(h->status, sizeof(int) * 4));
    TRY(ensure(h->ctr, sizeof(int) * 4));
    TRY(ensure(h->sd_buf, sizeof(SysDesc) * (size_t)B));
    TRY(ensure(h->blk_buf, sizeof(int) * h->h_blk.size()));
    TRY(ensure_atoms(h, N));
    TRY(ensure_host_e(h, B));
    // top-level Toeplitz tables g^{l-1} over all offsets (FP64), one per distinct top shape
    const double sc = ldexp(1.0, l - 1);
    for (const std::array<int, 4> &t : tops) {
        LevelGeom Lt;
        memset(&Lt, 0, sizeof Lt);
        for (int e = 0; e < 3; e++) Lt.n[e] = t[(size_t)e];
        TRY(launch_top_table(Lt, sc * h->p.a, sc * hh, h->ttop.as<double>() + t[3], st));
    }
    // lattice-cutoff weights W[n] = g^0(|n| h), |n| h < 2a, and the rows of the tap sphere
    if (grids && !h->stencil_ready) {
        int rad = 0;
        while ((double)(rad + 1) * hh < 2.0 * h->p.a) rad++;
        const int wd = 2 * rad + 1;
        std::vector<int4> rows;
        for (int dz = -rad; dz <= rad; dz++)
            for (int dy = -rad; dy <= rad; dy++) {
                int w = -1;
                for (int dx = rad; dx >= 0; dx--)
                    if (sqrt((double)(dx * dx + dy * dy + dz * dz)) * hh < 2.0 * h->p.a) { w = dx; break; }
                if (w >= 0) rows.push_back(make_int4(dy, dz, w, 0));
            }
        h->sg.rad = rad;
        h->sg.wdim = wd;
        h->sg.nrows = (int)rows.size();
        const size_t m = (size_t)wd * wd * wd;
        TRY(ensure(h->wst_d, sizeof(double) * m));
        TRY(ensure(h->wst_t, ts * m));
        TRY(ensure(h->rows, sizeof(int4) * rows.size()));
        TRY(launch_stencil_table(h->p.a, hh, rad, h->wst_d.as<double>(), st));
        if (h->precision == MSM_FP32) TRY(launch_cast_f64((int)m, h->wst_d.as<double>(), h->wst_t.as<float>(), st));
        else CUDA_TRY(cudaMemcpyAsync(h->wst_t.p, h->wst_d.p, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(h->rows.p, rows.data(), sizeof(int4) * rows.size(), cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));      // rows lives on the host stack
        h->stencil_ready = true;
    }
    h->sg.plane = 1;
    for (const SysDesc &D : d)
        for (int k = 0; k + 1 < l; k++) h->sg.plane = std::max(h->sg.plane, stencil_plane_values(D.gg.L[k], h->sg.rad));
    h->hsd.swap(d);
    if (grids && l > 1) {
        // descriptors of every (system, level) plane source: the grid buffer and the
        // geometry are fixed until the next change of batch
        h->st_maps.resize((size_t)B * (l - 1));
        if (h->precision == MSM_FP32)
            TRY(encode_stencil_maps<float>(h->hsd.data(), B, l - 1, h->sg.rad, h->qgrid.as<float>(), h->st_maps.data()));
        else
            TRY(encode_stencil_maps<double>(h->hsd.data(), B, l - 1, h->sg.rad, h->qgrid.as<double>(),
                                            h->st_maps.data()));
    }
    CUDA_TRY(cudaMemcpyAsync(h->sd_buf.p, h->hsd.data(), sizeof(SysDesc) * (size_t)B, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->blk_buf.p, h->h_blk.data(), sizeof(int) * h->h_blk.size(), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));          // the host copies may change with the next batch

    h->B = B;
    h->N = (int)N; h->M = (int)M; h->G = (int)G; h->UT = (int)UT; h->TT = (int)TT; h->PB = (int)PB;
    h->stiles = (int)ST;
    h->cp_cols = (int)CC;
    h->cp_max_cols = (int)CMAX;
    h->cp_max_icl = (int)CI;
    h->max_n = h->max_mol = h->max_units = h->max_bricks = h->max_atiles = h->max_top = h->max_lj_bricks = 0;
    for (int k = 0; k < MSM_MAX_LEVELS; k++) h->max_lev[k] = 0;
    for (const SysDesc &D : h->hsd) {
        h->max_n = std::max(h->max_n, D.n);
        h->max_mol = std::max(h->max_mol, D.n_mol);
        h->max_units = std::max(h->max_units, D.n_mol + (D.n - 3 * D.n_mol));
        h->max_bricks = std::max(h->max_bricks, D.nbricks);
        h->max_lj_bricks = std::max(h->max_lj_bricks, D.lj_nbricks);
        if (!grids) continue;
        h->max_atiles = std::max(h->max_atiles, anterp_tiles(D.gg.L[0]));
        for (int k = 0; k < l; k++) h->max_lev[k] = std::max(h->max_lev[k], D.gg.L[k].n[0] * D.gg.L[k].n[1] * D.gg.L[k].n[2]);
    }
    h->max_top = h->max_lev[l - 1];
    const SysDesc &D0 = h->hsd[0];
    h->cg = D0.g;
    h->gg = D0.gg;
    h->inv_h = D0.inv_h;
    memcpy(h->box, sys[0].box, sizeof h->box);
    for (int k = 0; k < 3; k++) { h->bd[k] = D0.bd[k]; h->nb[k] = D0.nb[k]; }
    h->nbricks = D0.nbricks;
    h->last_n = sys[0].n;
    h->sys_key.assign(sys, sys + B);
    h->tune_pending = pending;
    h->have_geom = true;
    h->geom_gen++;
    return MSM_OK;
}

static int ensure_atoms(msm_handle *h, int64_t n)
{
    const size_t ts = h->precision == MSM_FP32 ? sizeof(float) : sizeof(double);
    const size_t nn = (size_t)(n > 0 ? n : 1);
    TRY(ensure(h->key, sizeof(int) * nn));
    TRY(ensure(h->perm, sizeof(int) * nn));
    TRY(ensure(h->akey, sizeof(int) * nn));
    TRY(ensure(h->aflag, sizeof(int) * nn));
    TRY(ensure(h->rel, 4 * ts * nn));
    TRY(ensure(h->frac, 4 * ts * nn));
    TRY(ensure(h->apos, 4 * ts * nn));
    TRY(ensure(h->afrac, 4 * ts * nn));
    TRY(ensure(h->aw, 12 * ts * nn));
    TRY(ensure(h->sr, 4 * ts * nn));
    if (h->p.model == MSM_MODEL_WATER) {
        TRY(ensure(h->lj, 4 * ts * nn));
        TRY(ensure(h->lj_apos, 4 * ts * nn));
        TRY(ensure(h->lj_flag, sizeof(int) * nn));
        TRY(ensure(h->lj_perm, sizeof(int) * nn));
    }
    TRY(ensure(h->eatom, sizeof(double) * nn));
    TRY(ensure(h->vatom, sizeof(double) * nn));
    TRY(ensure(h->kin, sizeof(double) * nn));
    if (h->p.mts_steps > 1) TRY(ensure(h->eslow, sizeof(double) * nn));
    return MSM_OK;
}

static Batch batch_of(const msm_handle *h) { return Batch{h->B, h->sd_buf.as<SysDesc>()}; }

// Arguments of the short-range kernels for the current batch.
template <typename T>
static ShortArgs<T> short_args(msm_handle *h)
{
    ShortArgs<T> s;
    s.bt = batch_of(h);
    s.max_bricks = h->max_bricks;
    s.start = h->start.as<int>(); s.apos = h->apos.as<vec4<T>>(); s.aflag = h->aflag.as<int>();
    const double a = h->p.a;
    s.a = (T)a; s.a2 = (T)(a * a); s.a_sel = (T)(a + 1e-3 * h->p.h);
    if (h->p.method == MSM_METHOD_MSM) {
        s.c0 = (T)(GAMMA_C0 / a); s.c1 = (T)(GAMMA_C1 / (a * a * a)); s.c2 = (T)(GAMMA_C2 / (a * a * a * a * a));
        s.d0 = (T)(-2.5 / (a * a * a)); s.d1 = (T)(1.5 / (a * a * a * a * a));
    } else {                                               // pair term 1/r (Wolf: its own instance)
        s.c0 = s.c1 = s.c2 = s.d0 = s.d1 = T(0);
    }
    const double al = h->p.wolf_alpha;
    s.wolf = h->p.method == MSM_METHOD_WOLF;
    s.w_alpha = (T)al; s.w_shift = (T)(erfc(al * a) / a); s.w_c = (T)(2.0 * al / sqrt(M_PI));
    const double sg2 = h->p.lj_sigma * h->p.lj_sigma;
    const double sa6 = pow(sg2 / (a * a), 3.0);
    s.lj_s2 = (T)sg2; s.lj_4eps = (T)(4.0 * h->p.lj_epsilon); s.lj_24eps = (T)(24.0 * h->p.lj_epsilon);
    s.lj_shift = (T)(4.0 * h->p.lj_epsilon * (sa6 * sa6 - sa6));
    s.perm = h->perm.as<int>();
    s.sr = h->sr.as<vec4<T>>();
    s.lj = h->p.model == MSM_MODEL_WATER ? h->lj.as<vec4<T>>() : nullptr;
    s.cnt = nullptr;
    s.vl_ctl = nullptr;
    s.status = h->status.as<int>();
    s.scalar_pairs = (h->p.flags & MSM_FLAG_SCALAR_PAIRS) != 0;
    s.gcol = nullptr;
    s.gslot = nullptr;
    return s;
}

// Arguments of the cluster-pair kernels: the short-range constants and outputs of s.
static ClusterArgs cluster_args(msm_handle *h, const ShortArgs<float> &s)
{
    ClusterArgs c;
    c.bt = s.bt;
    c.max_cols = h->cp_max_cols; c.n_cols = h->cp_cols; c.max_icl = h->cp_max_icl;
    c.start = s.start; c.apos = s.apos; c.aflag = s.aflag; c.perm = s.perm;
    c.col_n = h->cp_coln.as<int>(); c.col_cl = h->cp_colcl.as<int>(); c.bsum = h->cp_bsum.as<int>();
    c.zc = h->cp_zc.as<int>();
    c.cpos = h->cp_pos.as<vec4<float>>(); c.cmol = h->cp_mol.as<int>(); c.cslot = h->cp_slot.as<int>();
    c.cbox = h->cp_box.as<vec4<float>>();
    c.a = s.a; c.a2 = s.a2; c.a_sel = s.a_sel;
    c.c0 = s.c0; c.c1 = s.c1; c.c2 = s.c2; c.d0 = s.d0; c.d1 = s.d1;
    c.sr = s.sr; c.lj = s.lj; c.vl_ctl = s.vl_ctl; c.status = s.status;
    return c;
}

// The brick autotuner: on the first evaluation of a geometry, time the
// short-range kernel for the five brick shapes around the heuristic's choice
// (after binning, on the real atoms; in a batch, one shape for all systems
// without a tuned entry, on the batched launch) and keep the fastest; for the
// water model, likewise the bricks of the LJ pass over the LJ-site list.  It runs
// outside any graph capture and synchronises the stream.
template <typename T>
static int autotune_bricks(msm_handle *h, cudaStream_t st)
{
    h->tune_pending = false;
    const int B = h->B;
    // the systems without a tuned entry (set_batch gave them the heuristic's bricks) are
    // tuned together: one shape for all of them, timed on the batched launch
    std::vector<int> todo;
    int big = -1;
    for (int b = 0; b < B; b++) {
        const SysDesc &D = h->hsd[(size_t)b];
        if (D.n > 0 && !find_tuned(h, D.n, D.g)) {
            todo.push_back(b);
            if (big < 0 || D.n > h->hsd[(size_t)big].n) big = b;
        }
    }
    if (todo.empty()) return MSM_OK;
    const bool model = h->p.model == MSM_MODEL_WATER;
    const int *status = h->status.as<int>();
    auto upload = [&]() {
        return cudaMemcpyAsync(h->sd_buf.p, h->hsd.data(), sizeof(SysDesc) * (size_t)B, cudaMemcpyHostToDevice, st);
    };
    auto most = [&](bool lj) {
        int m = 0;
        for (const SysDesc &D : h->hsd) m = std::max(m, lj ? D.lj_nbricks : D.nbricks);
        return m;
    };
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // time one configuration: the faster of two launches after a warm one
    auto timed = [&](const ShortArgs<T> &a, bool lj, float *ms) -> int {
        TRY(lj ? launch_short_lj<T>(a, st) : launch_short<T>(a, model, st));
        *ms = 1e30f;
        for (int rep = 0; rep < 2; rep++) {
            CUDA_TRY(cudaEventRecord(e0, st));
            TRY(lj ? launch_short_lj<T>(a, st) : launch_short<T>(a, model, st));
            CUDA_TRY(cudaEventRecord(e1, st));
            CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0;
            CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            *ms = std::min(*ms, t);
        }
        return MSM_OK;
    };
    const SysDesc &R = h->hsd[(size_t)big];
    auto build_lj_list = [&]() -> int {
        TRY(launch_lj_count<T>(h->M, h->start.as<int>(), h->aflag.as<int>(), h->lj_count.as<int>(), status, st));
        TRY(launch_scan(h->M, h->lj_count.as<int>(), h->lj_start.as<int>(), h->bsum.as<int>(), status, st));
        TRY(launch_lj_compact<T>(h->M, h->start.as<int>(), h->lj_start.as<int>(), h->apos.as<vec4<T>>(),
                                 h->aflag.as<int>(), h->perm.as<int>(), h->lj_apos.as<vec4<T>>(),
                                 h->lj_flag.as<int>(), h->lj_perm.as<int>(), status, st));
        return MSM_OK;
    };
    auto lj_args = [&]() {
        ShortArgs<T> sl = short_args<T>(h);
        sl.start = h->lj_start.as<int>(); sl.apos = h->lj_apos.as<vec4<T>>(); sl.aflag = h->lj_flag.as<int>();
        sl.perm = h->lj_perm.as<int>();
        return sl;
    };
    if (h->gp_on) {
        // i groups: the column width of the density heuristic and one narrower and one
        // wider, each timed with its group build; for the water model likewise the LJ
        // sites' groups on the LJ-site list
        auto timed_groups = [&](bool lj, float *ms) -> int {
            ShortArgs<T> a = lj ? lj_args() : short_args<T>(h);
            a.gcol = (lj ? h->lgp_col : h->gp_col).template as<int>();
            a.gslot = (lj ? h->lgp_slot : h->gp_slot).template as<int>();
            a.max_bricks = lj ? h->lgp_max_groups : h->gp_max_groups;
            auto run = [&]() -> int {
                if (lj)
                    TRY(launch_groups<T>(a.bt, true, h->lgp_max_cols, h->gp_max_nz, h->lgp_cols, a.start, a.apos,
                                         h->lgp_cnt.as<int>(), h->lgp_col.as<int>(), h->lgp_bsum.as<int>(),
                                         h->lgp_slot.as<int>(), status, st));
                else
                    TRY(launch_groups<T>(a.bt, false, h->gp_max_cols, h->gp_max_nz, h->gp_cols, a.start, a.apos,
                                         h->gp_cnt.as<int>(), h->gp_col.as<int>(), h->gp_bsum.as<int>(),
                                         h->gp_slot.as<int>(), status, st));
                return lj ? launch_short_lj<T>(a, st) : launch_short<T>(a, model, st);
            };
            TRY(run());
            *ms = 1e30f;
            for (int rep = 0; rep < 2; rep++) {
                CUDA_TRY(cudaEventRecord(e0, st));
                TRY(run());
                CUDA_TRY(cudaEventRecord(e1, st));
                CUDA_TRY(cudaEventSynchronize(e1));
                float t = 0;
                CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
                *ms = std::min(*ms, t);
            }
            return MSM_OK;
        };
        auto tune_width = [&](bool lj) -> int {
            const SysDesc &Rc = h->hsd[(size_t)big];
            const int w0 = lj ? Rc.lgp_cw : Rc.gp_cw;
            float best = 1e30f;
            int best_w = w0;
            for (int w = std::max(1, w0 - 1); w <= std::min(8, w0 + 1); w++) {
                for (int b : todo) (lj ? h->hsd[(size_t)b].lgp_cw : h->hsd[(size_t)b].gp_cw) = w;
                TRY(layout_groups(h, h->hsd));
                CUDA_TRY(upload());
                float ms;
                TRY(timed_groups(lj, &ms));
                if (ms < best) { best = ms; best_w = w; }
            }
            for (int b : todo) (lj ? h->hsd[(size_t)b].lgp_cw : h->hsd[(size_t)b].gp_cw) = best_w;
            TRY(layout_groups(h, h->hsd));
            CUDA_TRY(upload());
            return MSM_OK;
        };
        TRY(tune_width(false));
        if (model) {
            TRY(build_lj_list());
            TRY(tune_width(true));
        }
    } else {
        const int h0 = brick_heuristic(R.n, R.g);
        float best = 1e30f;
        int best_s = h0;
        for (int sidx = std::max(0, h0 - 2); sidx <= std::min(kNumShapes - 1, h0 + 2); sidx++) {
            for (int b : todo) set_bricks(h->hsd[(size_t)b], kBrickShapes[sidx]);
            CUDA_TRY(upload());
            ShortArgs<T> sa = short_args<T>(h);
            sa.max_bricks = most(false);
            float ms;
            TRY(timed(sa, false, &ms));
            if (ms < best) { best = ms; best_s = sidx; }
        }
        for (int b : todo) set_bricks(h->hsd[(size_t)b], kBrickShapes[best_s]);
        CUDA_TRY(upload());
        int best_l = 0;
        if (model) {
            // the LJ pass's bricks likewise, on the LJ-site list the evaluation builds next
            TRY(build_lj_list());
            ShortArgs<T> sl = lj_args();
            const int l0 = brick_heuristic(R.n_mol + (R.n - 3 * R.n_mol), R.g);
            float best_lj = 1e30f;
            best_l = l0;
            for (int sidx = std::max(0, l0 - 2); sidx <= std::min(kNumShapes - 1, l0 + 2); sidx++) {
                for (int b : todo) set_lj_bricks(h->hsd[(size_t)b], kBrickShapes[sidx]);
                CUDA_TRY(upload());
                sl.max_bricks = most(true);
                float ms;
                TRY(timed(sl, true, &ms));
                if (ms < best_lj) { best_lj = ms; best_l = sidx; }
            }
            for (int b : todo) set_lj_bricks(h->hsd[(size_t)b], kBrickShapes[best_l]);
            CUDA_TRY(upload());
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_TRY(cudaStreamSynchronize(st));
    for (int b : todo) {
        const SysDesc &D = h->hsd[(size_t)b];
        Tuned t;
        t.n = D.n;
        for (int k = 0; k < 3; k++) {
            t.nc[k] = D.g.nc[k];
            t.bd[k] = D.bd[k];
            t.lj_bd[k] = model ? D.lj_bd[k] : 0;
        }
        t.gcw = h->gp_on ? D.gp_cw : 0;
        t.lgcw = (h->gp_on && model) ? D.lgp_cw : 0;
        h->tuned.push_back(t);
    }
    h->max_bricks = most(false);
    h->max_lj_bricks = most(true);
    const SysDesc &D0 = h->hsd[0];
    for (int k = 0; k < 3; k++) { h->bd[k] = D0.bd[k]; h->nb[k] = D0.nb[k]; }
    h->nbricks = D0.nbricks;
    h->geom_gen++;
    return MSM_OK;
}

// One evaluation of the current batch on device arrays (systems concatenated).
// eatom/vatom get per-atom energy and virial; sums[4 s + 0] = U_s,
// sums[4 s + 1] = virial_s.  No host synchronisation (except the autotuner's,
// once per geometry).
// Evaluation modes (multiple time stepping): the whole force into forces; the
// split into fast (forces) and slow (fslow) parts; or the fast part alone.
enum EvalMode { EVAL_FULL = 0, EVAL_SPLIT = 1, EVAL_FAST = 2 };

struct EvalIO {
    const double *pos, *q;
    const uint8_t *lj;       // nullable (device)
    double *forces, *pot;    // device, nullable
    double *fslow = nullptr; // EVAL_SPLIT: slow forces (device)
    int mode = EVAL_FULL;
};

template <typename T>
static int evaluate_t(msm_handle *h, const EvalIO &io, cudaStream_t st)
{
    int *status = h->status.as<int>();
    const bool model = h->p.model == MSM_MODEL_WATER;
    const Batch bt = batch_of(h);

    BinArgs<T> b;
    b.bt = bt; b.n_total = h->N; b.m_total = h->M; b.max_n = h->max_n;
    b.pos = io.pos; b.q = io.q; b.lj = io.lj;
    b.key = h->key.as<int>(); b.count = h->count.as<int>(); b.start = h->start.as<int>(); b.perm = h->perm.as<int>();
    b.bsum = h->bsum.as<int>(); b.rel = h->rel.as<vec4<T>>(); b.frac = h->frac.as<vec4<T>>();
    b.apos = h->apos.as<vec4<T>>(); b.afrac = h->afrac.as<vec4<T>>(); b.akey = h->akey.as<int>();
    b.aflag = h->aflag.as<int>(); b.aw = h->aw.as<vec4<T>>(); b.status = status;
    { PROF(ST_BIN); TRY(launch_bin<T>(b, st)); }
    if (h->tune_pending) TRY(autotune_bricks<T>(h, st));

    // The grid chain (steps 2-7) depends on the binning only, the short range (step 1)
    // likewise; interpolation needs both.  Unless the stages are being timed one by one
    // (or Verlet lists are on), the grid chain runs on a second, high-priority stream
    // forked here and joined before interpolation: its small, latency-bound launches
    // (the lattice cutoff keeps about four CTAs per SM busy) fill the SMs beside the
    // issue-bound pair kernels.
    const bool grids = has_grids(h->p) && io.mode != EVAL_FAST;
    const bool split = grids && io.mode == EVAL_SPLIT;
    const bool fork = grids && !h->prof.on && !h->list_on;
    cudaStream_t gs = st;
    if (fork) {
        if (!h->grid_st) {
            int lo = 0, hi = 0;
            CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            CUDA_TRY(cudaStreamCreateWithPriority(&h->grid_st, cudaStreamNonBlocking, hi));
            CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
            CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        CUDA_TRY(cudaEventRecord(h->ev_fork, st));
        CUDA_TRY(cudaStreamWaitEvent(h->grid_st, h->ev_fork, 0));
        gs = h->grid_st;
    }
    T *qg = h->qgrid.as<T>(), *uc = h->ucut.as<T>(), *ug = h->ugrid.as<T>();
    if (grids) {
        cudaStream_t st = gs;                                  // the grid chain's stream
        // step 2: anterpolation
        AnterpArgs<T> an;
        an.bt = bt; an.max_tiles = h->max_atiles; an.n_total = (int)h->N; an.start = h->start.as<int>();
        an.aw = h->aw.as<vec4<T>>();
        an.q = qg; an.status = status;
        { PROF(ST_ANTERP); TRY(launch_anterp<T>(an, st)); }

        // steps 3-4: restriction down the levels, then the lattice cutoff of levels 0..l-2 in one launch
        const int l = h->p.n_levels;
        {
            PROF(ST_RESTRICT);
            for (int k = 0; k + 1 < l; k++) TRY(launch_restrict<T>(bt, k, h->max_lev[k + 1], qg, status, st));
        }
        if (l > 1) {
            StencilArgs<T> sa;
            sa.bt = bt; sa.nlev = l - 1; sa.blk_off = h->blk_buf.as<int>(); sa.total_tiles = h->stiles; sa.sg = h->sg;
            sa.w = h->wst_t.as<T>(); sa.rows = h->rows.as<int4>(); sa.q = qg; sa.ucut = uc; sa.ucut_len = (size_t)h->G;
            sa.status = status;
            PROF(ST_STENCIL);
            TRY(launch_stencil<T>(sa, h->st_maps.data(), h->h_blk.data(), h->status.as<int>() + 2, st));
        }
        // step 5: top level in FP64
        { PROF(ST_TOP); TRY(launch_top<T>(bt, h->max_top, h->ttop.as<double>(), qg, h->utop.as<double>(), status, st)); }
        // steps 6-7: prolongation back to level 0
        {
            PROF(ST_PROLONG);
            if (l == 1) {
                TRY(launch_top_to_grid<T>(bt, h->max_top, h->utop.as<double>(), ug, status, st));
            } else {
                TRY(launch_prolong<T>(bt, l - 2, h->max_lev[l - 2], uc, h->utop.as<double>(), true, ug, status, st));
                for (int k = l - 3; k >= 0; k--)
                    TRY(launch_prolong<T>(bt, k, h->max_lev[k], uc, h->utop.as<double>(), false, ug, status, st));
            }
        }
    }

    // step 1: short range
    ShortArgs<T> s = short_args<T>(h);
    if (h->gp_on && !(sizeof(T) == sizeof(float) && h->cp_on)) {
        // i groups of the Coulomb pass (after the binning: they read the cell starts; the
        // cluster-pair pass, when on, replaces it)
        TRY(launch_groups<T>(s.bt, false, h->gp_max_cols, h->gp_max_nz, h->gp_cols, s.start, s.apos,
                             h->gp_cnt.as<int>(), h->gp_col.as<int>(), h->gp_bsum.as<int>(), h->gp_slot.as<int>(),
                             s.status, st));
        s.gcol = h->gp_col.as<int>();
        s.gslot = h->gp_slot.as<int>();
        s.max_bricks = h->gp_max_groups;
    }
    // the lists address the bricks they were built for: never use them on another brick set
    if (h->list_on && h->nbricks != h->vl_nbricks) h->list_on = false;
    s.vl_ctl = h->list_on ? h->vl_ctl.as<int>() : nullptr;
    {
        ListArgs<T> la;
        if (h->list_on) {
            const double a = h->p.a;
            la.g = h->cg;
            for (int d = 0; d < 3; d++) { la.bd[d] = h->bd[d]; la.nb[d] = h->nb[d]; }
            la.nbricks = h->nbricks;
            la.cap = h->vl_cap; la.cap_lj = h->vl_cap_lj;
            const double rl = a + h->p.list_skin;
            la.a2 = s.a2; la.rl2 = (T)(rl * rl); la.rl_sel = (T)(rl + 1e-3 * h->p.h);
            la.skin_half2 = (T)(0.25 * h->p.list_skin * h->p.list_skin);
            la.c0 = s.c0; la.c1 = s.c1; la.c2 = s.c2; la.d0 = s.d0; la.d1 = s.d1;
            la.lj_s2 = s.lj_s2; la.lj_4eps = s.lj_4eps; la.lj_24eps = s.lj_24eps; la.lj_shift = s.lj_shift;
            la.model = model; la.n = h->N; la.x = io.pos; la.q = io.q;
            la.perm = h->perm.as<int>(); la.start = h->start.as<int>(); la.apos = h->apos.as<vec4<T>>();
            la.aflag = h->aflag.as<int>();
            la.vl_perm = h->vl_perm.as<int>(); la.vl_start = h->vl_start.as<int>(); la.vl_xref = h->vl_xref.as<double>();
            la.vl_pos = h->vl_pos.as<vec4<T>>(); la.rtab = h->vl_rtab.as<int>(); la.rtn = h->vl_rtn.as<int>();
            la.cnt = h->vl_cnt.as<int>(); la.cntlj = h->vl_cntlj.as<int>();
            la.nbr = h->vl_nbr.as<unsigned long long>(); la.nbr_lj = h->vl_nbr_lj.as<unsigned long long>();
            la.ctl = h->vl_ctl.as<int>(); la.sr = s.sr; la.lj = s.lj; la.status = status;
            PROF(ST_LIST);
            TRY(launch_list_maintain<T>(la, st));
        }
        {
            PROF(ST_SHORT);
            if (h->list_on) TRY(launch_list_force<T>(la, st));
            if constexpr (sizeof(T) == sizeof(float)) {
                if (h->cp_on) {
                    const ClusterArgs ca = cluster_args(h, s);
                    TRY(launch_cluster_build(ca, model, st));
                    TRY(launch_cluster_short(ca, model, st));
                } else {
                    TRY(launch_short<T>(s, model, st));
                }
            } else {
                TRY(launch_short<T>(s, model, st));
            }
        }
        if (model) {
            PROF(ST_LJ);
            // O-O Lennard-Jones over the LJ sites alone
            TRY(launch_lj_count<T>(h->M, h->start.as<int>(), h->aflag.as<int>(), h->lj_count.as<int>(), status, st));
            TRY(launch_scan(h->M, h->lj_count.as<int>(), h->lj_start.as<int>(), h->bsum.as<int>(), status, st));
            TRY(launch_lj_compact<T>(h->M, h->start.as<int>(), h->lj_start.as<int>(), h->apos.as<vec4<T>>(),
                                     h->aflag.as<int>(), h->perm.as<int>(), h->lj_apos.as<vec4<T>>(),
                                     h->lj_flag.as<int>(), h->lj_perm.as<int>(), status, st));
            ShortArgs<T> sl = s;
            sl.max_bricks = h->max_lj_bricks;
            sl.start = h->lj_start.as<int>(); sl.apos = h->lj_apos.as<vec4<T>>(); sl.aflag = h->lj_flag.as<int>();
            sl.perm = h->lj_perm.as<int>();
            if (h->gp_on) {
                TRY(launch_groups<T>(sl.bt, true, h->lgp_max_cols, h->gp_max_nz, h->lgp_cols, sl.start, sl.apos,
                                     h->lgp_cnt.as<int>(), h->lgp_col.as<int>(), h->lgp_bsum.as<int>(), h->lgp_slot.as<int>(), status, st));
                sl.gcol = h->lgp_col.as<int>();
                sl.gslot = h->lgp_slot.as<int>();
                sl.max_bricks = h->lgp_max_groups;
            }
            TRY(launch_short_lj<T>(sl, st));
        }
    }

    if (fork) {
        CUDA_TRY(cudaEventRecord(h->ev_join, gs));
        CUDA_TRY(cudaStreamWaitEvent(st, h->ev_join, 0));
    }

    // step 8-9: interpolation, totals, scatter to the caller's order
    InterpArgs<T> ia;
    ia.bt = bt; ia.max_n = h->max_n; ia.perm = h->perm.as<int>(); ia.akey = h->akey.as<int>();
    ia.afrac = h->afrac.as<vec4<T>>(); ia.sr = h->sr.as<vec4<T>>(); ia.lj = model ? h->lj.as<vec4<T>>() : nullptr;
    ia.u = grids ? ug : nullptr; ia.pos = io.pos; ia.q = io.q; ia.ke = h->p.coulomb_k;
    // self coefficient: phi_i -= q_i self (the MSM's gamma(0)/a; Wolf's neutralisation term)
    const double al = h->p.wolf_alpha, a_ = h->p.a;
    // (a fast-only evaluation has no self term: it belongs to the slow, grid part)
    ia.self = io.mode == EVAL_FAST ? 0.0
            : h->p.method == MSM_METHOD_MSM ? GAMMA_C0 / a_
            : h->p.method == MSM_METHOD_WOLF ? erfc(al * a_) / a_ + 2.0 * al / sqrt(M_PI) : 0.0;
    ia.wall_k = model ? h->p.wall_k : 0.0; ia.wall_w = h->p.wall_width;
    ia.forces = io.forces; ia.pot = io.pot; ia.eatom = h->eatom.as<double>(); ia.vatom = h->vatom.as<double>();
    ia.fslow = split ? io.fslow : nullptr; ia.eslow = split ? h->eslow.as<double>() : nullptr;
    ia.status = status;
    { PROF(ST_INTERP); TRY(launch_interp<T>(ia, st)); }
    PROF(ST_SUMS);
    if (model && grids && h->max_mol > 0) {           // the cutoff methods skipped these pairs outright
        ExclArgs ex;
        ex.bt = bt; ex.max_mol = h->max_mol; ex.x = io.pos; ex.q = io.q; ex.ke = h->p.coulomb_k; ex.a = h->p.a;
        ex.inv_a = 1.0 / h->p.a;
        ex.forces = io.forces; ex.pot = io.pot; ex.eatom = h->eatom.as<double>(); ex.vatom = h->vatom.as<double>();
        ex.fslow = ia.fslow; ex.eslow = ia.eslow;
        ex.status = status;
        TRY(launch_exclusions<T>(ex, st));
    }
    // sums[s][0] energy, [1] virial, [2] slow energy (split evaluations only: a
    // fast-only evaluation leaves the last one in place)
    const double *cols[3] = {h->eatom.as<double>(), h->vatom.as<double>(), h->eslow.as<double>()};
    TRY(launch_sum(bt, h->max_n, h->PB, split ? 3 : 2, cols, h->partials.as<double>(), h->sums.as<double>(), 4,
                   status, st));
    return MSM_OK;
}

static int evaluate(msm_handle *h, const EvalIO &io, int B, const SysIn *sys, cudaStream_t st)
{
    if (h->p.model != MSM_MODEL_WATER)
        for (int s = 0; s < B; s++)
            if (sys[s].n_mol) return fail_msg(MSM_EINVAL, "rigid molecules need the water model");
    TRY(set_batch(h, B, sys, st));
    CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, st));
    if (h->precision == MSM_FP32) return evaluate_t<float>(h, io, st);
    return evaluate_t<double>(h, io, st);
}

static int list_grow(msm_handle *h, cudaStream_t st);

// Copy the device status word to the host, synchronise, translate.
static int finish(msm_handle *h, cudaStream_t st)
{
    CUDA_TRY(cudaMemcpyAsync(h->h_status, h->status.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
    if (h->vl_ctl.p) CUDA_TRY(cudaMemcpyAsync(h->h_ctl, h->vl_ctl.p, sizeof(int) * 8, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    prof_resolve(h);
    if (h->vl_ctl.p) {
        h->vl_builds += h->h_ctl[7];
        h->vl_overflows += h->h_ctl[1] ? 1 : 0;
        for (int k = 4; k <= 6; k++) h->vl_seen[k - 4] = std::max(h->vl_seen[k - 4], (int64_t)h->h_ctl[k]);
        if (h->h_ctl[7]) CUDA_TRY(cudaMemsetAsync(h->vl_ctl.as<int>() + 7, 0, sizeof(int), st));
        if (h->h_ctl[1]) TRY(list_grow(h, st));
    }
    const int s = h->h_status[0];
    if (s == MSM_ENOCONV && h->h_status[1])
        return fail_msg(s, "%s did not converge (molecule starting at atom %d of the batch)",
                        h->h_status[1] == 1 ? "SHAKE" : "RATTLE", h->h_status[3] - 1);
    if (s != 0) return fail_msg(s, "%s", status_text(s));
    return MSM_OK;
}

// Stage an input array on the device if it lives in host memory.
static int stage_in(DevBuf &buf, const void *src, size_t bytes, const void **dev, cudaStream_t st)
{
    if (!src || on_device(src)) { *dev = src; return MSM_OK; }
    TRY(ensure(buf, bytes));
    CUDA_TRY(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = buf.p;
    return MSM_OK;
}

// Per-system column c of sums (stride 4) to dst[0..B-1] (device or host).
static int copy_sums(double *dst, const msm_handle *h, int c, cudaStream_t st)
{
    if (!dst) return MSM_OK;
    CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(double), h->sums.as<double>() + c, 4 * sizeof(double), sizeof(double),
                               (size_t)h->B, cudaMemcpyDefault, st));
    return MSM_OK;
}

// One evaluation of B systems whose per-atom arrays are concatenated.
static int forces_impl(msm_handle *h, int B, const SysIn *sys, const double *pos, const double *q,
                       const uint8_t *lj, double *energies, double *forces, double *pot, double *virials,
                       cudaStream_t st)
{
    if (!h) return fail_msg(MSM_EINVAL, "handle is NULL");
    int64_t n = 0;
    for (int s = 0; s < B; s++) {
        if (sys[s].n < 0) return fail_msg(MSM_EINVAL, "n < 0");
        n += sys[s].n;
    }
    if (n > 0 && (!pos || !q)) return fail_msg(MSM_EINVAL, "pos and q are required");
    TRY(check_arrays({pos, q, lj, energies, forces, pot, virials}));
    const size_t nn = (size_t)n;
    EvalIO io;
    const void *dp, *dq, *dl;
    TRY(stage_in(h->in_pos, pos, sizeof(double) * 3 * nn, &dp, st));
    TRY(stage_in(h->in_q, q, sizeof(double) * nn, &dq, st));
    TRY(stage_in(h->in_lj, lj, nn, &dl, st));
    io.pos = (const double *)dp; io.q = (const double *)dq; io.lj = (const uint8_t *)dl;
    const bool f_host = forces && !on_device(forces), p_host = pot && !on_device(pot);
    if (f_host) TRY(ensure(h->out_f, sizeof(double) * 3 * nn));
    if (p_host) TRY(ensure(h->out_p, sizeof(double) * nn));
    io.forces = f_host ? h->out_f.as<double>() : forces;
    io.pot = p_host ? h->out_p.as<double>() : pot;
    TRY(evaluate(h, io, B, sys, st));
    if (f_host && n > 0) CUDA_TRY(cudaMemcpyAsync(forces, h->out_f.p, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (p_host && n > 0) CUDA_TRY(cudaMemcpyAsync(pot, h->out_p.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, st));
    TRY(copy_sums(energies, h, 0, st));
    TRY(copy_sums(virials, h, 1, st));
    return finish(h, st);
}

extern "C" int msm_energy_forces(msm_handle *h, int64_t n, const double *pos, const double *q, const double box[6],
                                 double *energy, double *forces, double *potentials, double *virial, void *stream)
{
    if (h && h->p.model != MSM_MODEL_CHARGES)
        return fail_msg(MSM_EINVAL, "msm_energy_forces evaluates point charges; use msm_system_forces for the water model");
    if (!box) return fail_msg(MSM_EINVAL, "box is NULL");
    SysIn s;
    s.n = n; s.n_mol = 0;
    memcpy(s.box, box, sizeof s.box);
    return forces_impl(h, 1, &s, pos, q, nullptr, energy, forces, potentials, virial, (cudaStream_t)stream);
}

extern "C" int msm_system_forces(msm_handle *h, const msm_system *sys, double *energy, double *forces,
                                 double *potentials, void *stream)
{
    if (!sys) return fail_msg(MSM_EINVAL, "system is NULL");
    SysIn s;
    s.n = sys->n; s.n_mol = sys->n_mol;
    memcpy(s.box, sys->box, sizeof s.box);
    return forces_impl(h, 1, &s, sys->x, sys->q, sys->lj, energy, forces, potentials, nullptr, (cudaStream_t)stream);
}

extern "C" int msm_energy_forces_batched(msm_handle *h, int32_t n_sys, const int64_t *offsets, const double *pos,
                                         const double *q, const double *boxes, double *energies, double *forces,
                                         double *potentials, void *stream)
{
    if (!h || n_sys < 1 || !offsets || !boxes) return fail_msg(MSM_EINVAL, "bad batched arguments");
    if (h->p.model != MSM_MODEL_CHARGES) return fail_msg(MSM_EINVAL, "batched evaluation takes point charges");
    if (offsets[0] != 0) return fail_msg(MSM_EINVAL, "offsets must start at 0");
    std::vector<SysIn> sys((size_t)n_sys);
    for (int s = 0; s < n_sys; s++) {
        if (offsets[s + 1] < offsets[s]) return fail_msg(MSM_EINVAL, "offsets must be non-decreasing from 0");
        sys[(size_t)s].n = offsets[s + 1] - offsets[s];
        sys[(size_t)s].n_mol = 0;
        memcpy(sys[(size_t)s].box, boxes + 6 * s, sizeof sys[0].box);
    }
    return forces_impl(h, n_sys, sys.data(), pos, q, nullptr, energies, forces, potentials, nullptr,
                       (cudaStream_t)stream);
}

// ----------------------------------------------------------------- dynamics

// A batch of MD systems in concatenated device arrays.
struct RunSys {
    int B;
    const SysIn *sys;
    double *x, *v;
    const double *q, *m;
    const uint8_t *lj;
    double *f = nullptr;      // device forces carried in/out (nullable)
    bool f_valid = false;     // f and e0 hold F, U of the start positions
    const double *e0 = nullptr;   // host, B energies when f_valid
};

// ------------------------------------------------------------ Verlet lists

static int list_alloc(msm_handle *h, int64_t n, size_t vsz)
{
    const size_t nn = (size_t)(n > 0 ? n : 1);
    TRY(ensure(h->vl_perm, sizeof(int) * nn));
    TRY(ensure(h->vl_start, sizeof(int) * ((size_t)h->cg.ncells + 1)));
    TRY(ensure(h->vl_xref, sizeof(double) * 3 * nn));
    TRY(ensure(h->vl_pos, vsz * nn));
    TRY(ensure(h->vl_rtab, sizeof(int) * (size_t)VL_ROWS * (size_t)(h->vl_nbricks > 0 ? h->vl_nbricks : 1)));
    TRY(ensure(h->vl_rtn, sizeof(int) * (size_t)(h->vl_nbricks > 0 ? h->vl_nbricks : 1)));
    TRY(ensure(h->vl_cnt, sizeof(int) * nn));
    TRY(ensure(h->vl_cntlj, sizeof(int) * nn));
    TRY(ensure(h->vl_nbr, sizeof(uint16_t) * nn * (size_t)h->vl_cap));
    TRY(ensure(h->vl_nbr_lj, sizeof(uint16_t) * nn * (size_t)(h->vl_cap_lj > 0 ? h->vl_cap_lj : 4)));
    TRY(ensure(h->vl_ctl, sizeof(int) * 8));
    return MSM_OK;
}

static int list_invalidate(msm_handle *h, cudaStream_t st)
{
    CUDA_TRY(cudaMemsetAsync(h->vl_ctl.p, 0, sizeof(int) * 8, st));
    const int invalid = 1;
    CUDA_TRY(cudaMemcpyAsync(h->vl_ctl.as<int>() + 2, &invalid, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));                    // 'invalid' lives on the host stack
    return MSM_OK;
}

// Size the lists for a single system and invalidate them when the system
// changed or the call does not continue a trajectory (fresh): md_run's results
// then depend only on its inputs, never on what the handle ran before.
template <typename T>
static int list_setup(msm_handle *h, const RunSys &s, bool fresh, cudaStream_t st)
{
    TRY(set_batch(h, 1, s.sys, st));
    const SysIn &S = s.sys[0];
    const double rl = h->p.a + h->p.list_skin;
    const bool changed = S.n != h->vl_key_n || S.n_mol != h->vl_key_nmol || s.lj != h->vl_key_lj ||
                         memcmp(S.box, h->vl_key_box, sizeof h->vl_key_box) != 0 || h->nbricks != h->vl_nbricks;
    if (!changed && !fresh && h->vl_ctl.p) return MSM_OK;
    if (h->vl_cap == 0) {
        // entries per atom: pairs within a + skin at 1.3x the box's mean density
        const double vol = S.box[3] * S.box[4] * S.box[5];
        const double dens = (double)S.n / vol;
        const double want = 1.3 * dens * 4.18879020478639 * rl * rl * rl + 32.0;
        h->vl_cap = ((std::max(64, (int)want) + 3) / 4) * 4;
        h->vl_cap_lj = h->p.model == MSM_MODEL_WATER ? ((h->vl_cap / 2 + 3) / 4) * 4 : 4;
    }
    h->vl_nbricks = h->nbricks;
    TRY(list_alloc(h, S.n, sizeof(vec4<T>)));
    TRY(list_invalidate(h, st));
    h->vl_key_n = S.n; h->vl_key_nmol = S.n_mol; h->vl_key_lj = s.lj;
    memcpy(h->vl_key_box, S.box, sizeof h->vl_key_box);
    return MSM_OK;
}

// After an overflow: grow the exceeded capacity, invalidate, resume with lists
// next time; a brick the 16-bit entries cannot address (more than VL_ROWS rows
// or a row of VL_OFFS atoms or more) turns the lists off for this handle.
static int list_grow(msm_handle *h, cudaStream_t st)
{
    const int *c = h->h_ctl;
    const size_t vsz = h->precision == MSM_FP32 ? sizeof(vec4<float>) : sizeof(vec4<double>);
    bool grew = false;
    if (c[4] > h->vl_cap) { h->vl_cap = (((int)(1.2 * c[4]) + 16 + 3) / 4) * 4; grew = true; }
    if (c[5] > h->vl_cap_lj) { h->vl_cap_lj = (((int)(1.2 * c[5]) + 16 + 3) / 4) * 4; grew = true; }
    if (!grew) h->p.list_skin = 0.0;                        // not a capacity: cell search from now on
    TRY(list_alloc(h, h->vl_key_n, vsz));
    return list_invalidate(h, st);
}

template <typename T> static double shake_tol() { return sizeof(T) == 4 ? 2e-6 : 1e-12; }
template <typename T> static double rattle_tol() { return sizeof(T) == 4 ? 2e-6 : 1e-14; }

// (U, K) of every system into uk at the device step counter, then advance it.
// kin_ready: the per-atom kinetic energies are already in h->kin (written by
// the second half kick).
static int record_uk(msm_handle *h, const RunSys &s, double *uk, int64_t uk_stride, cudaStream_t st,
                     bool kin_ready = false, bool add_slow = false)
{
    if (!kin_ready) TRY(launch_kinetic(h->N, s.v, s.m, h->kin.as<double>(), st));
    const double *cols[1] = {h->kin.as<double>()};
    TRY(launch_sum(batch_of(h), h->max_n, h->PB, 1, cols, h->partials.as<double>(), h->kin_s.as<double>(), 1,
                   h->status.as<int>(), st));
    return launch_record_uk(h->B, h->sums.as<double>(), 4, h->kin_s.as<double>(), uk, (int)uk_stride,
                            h->ctr.as<int>(), add_slow, st);
}

// Fast steps per slow step (1: plain velocity Verlet).
static int mts_of(const msm_handle *h) { return h->p.mts_steps > 1 ? h->p.mts_steps : 1; }

// One velocity Verlet step of the batch: half kick + drift + SHAKE, forces,
// half kick + RATTLE (+ the energies when recorded).  With multiple time
// stepping, one outer step: k fast steps whose first and last half kicks add
// the slow force's impulse k dt/2 (io.fslow, weight k), fast-only evaluations
// inside, and a split evaluation (fast and slow parts) at the end.
template <typename T>
static int md_step(msm_handle *h, const RunSys &s, const EvalIO &io, const VVArgs &va, double *uk,
                   int64_t uk_stride, cudaStream_t st)
{
    const int k = mts_of(h);
    if (k == 1) {
        { PROF(ST_VV1); TRY(launch_vv_first<T>(va, st)); }
        TRY(evaluate_t<T>(h, io, st));
        { PROF(ST_VV2); TRY(launch_vv_second<T>(va, uk ? h->kin.as<double>() : nullptr, st)); }
        if (uk) TRY(record_uk(h, s, uk, uk_stride, st, true));
        return MSM_OK;
    }
    for (int j = 0; j < k; j++) {
        const bool first = j == 0, last = j == k - 1;
        VVArgs v1 = va;
        v1.fs = first ? io.fslow : nullptr; v1.ws = (double)k;
        { PROF(ST_VV1); TRY(launch_vv_first<T>(v1, st)); }
        EvalIO e = io;
        e.mode = last ? EVAL_SPLIT : EVAL_FAST;
        TRY(evaluate_t<T>(h, e, st));
        VVArgs v2 = va;
        v2.fs = last ? io.fslow : nullptr; v2.ws = (double)k;
        { PROF(ST_VV2); TRY(launch_vv_second<T>(v2, uk ? h->kin.as<double>() : nullptr, st)); }
        if (uk) TRY(record_uk(h, s, uk, uk_stride, st, true, !last));
    }
    return MSM_OK;
}

// Capture one md step (an outer step with multiple time stepping) into a CUDA
// graph on the handle's own stream (capture records the launches; nothing
// runs), or reuse the graph captured for the same arrays, geometry and buffers.
static GraphKey graph_key(const msm_handle *h, const RunSys &s, const EvalIO &io, double dt, double *uk,
                          int64_t uk_stride)
{
    GraphKey k;
    memset(&k, 0, sizeof k);
    k.x = s.x; k.v = s.v; k.f = io.forces; k.q = s.q; k.m = s.m; k.lj = s.lj; k.uk = uk;
    k.uk_stride = uk_stride; k.geom_gen = h->geom_gen; k.alloc_gen = g_alloc_gen.load(); k.dt = dt;
    k.B = s.B; k.list_on = h->list_on ? 1 : 0; k.mts = mts_of(h);
    return k;
}

template <typename T>
static int md_graph(msm_handle *h, const RunSys &s, const EvalIO &io, const VVArgs &va, double dt, double *uk,
                    int64_t uk_stride)
{
    const GraphKey k = graph_key(h, s, io, dt, uk, uk_stride);
    if (h->gexec && memcmp(&k, &h->gkey, sizeof k) == 0) return MSM_OK;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (!h->cap_st) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking));
    const long long l0 = g_launches.load();
    CUDA_TRY(cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeRelaxed));
    const int rc = md_step<T>(h, s, io, va, uk, uk_stride, h->cap_st);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(h->cap_st, &g);
    h->g_kernels = g_launches.load() - l0;
    g_launches.fetch_sub(h->g_kernels);                    // counted when replayed
    if (rc != MSM_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return fail_cuda(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    const cudaError_t e2 = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) { h->gexec = nullptr; return fail_cuda(e2, "cudaGraphInstantiate", __FILE__, __LINE__); }
    h->gkey = k;
    return MSM_OK;
}

// n_steps of velocity Verlet on a batch in device arrays; uk (device,
// nullable) gets (U, K) of system b before the first and after every step at
// uk[b * uk_stride + 2 * step].  With graphs on (and the profiler off) the
// steps replay one captured graph; the first step of a call runs launch by
// launch unless the graph cached by an earlier call was captured for the same
// arrays, geometry and buffers.  No host synchronisation.
template <typename T>
static int run_md_t(msm_handle *h, const RunSys &s, double dt, int n_steps, double *uk, int64_t uk_stride,
                    cudaStream_t st)
{
    int64_t n = 0;
    for (int b = 0; b < s.B; b++) n += s.sys[b].n;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const int k = mts_of(h);                            // fast steps per slow step
    if (n_steps % k) return fail_msg(MSM_EINVAL, "n_steps (%d) must be a multiple of mts_steps (%d)", n_steps, k);
    TRY(ensure(h->md_xo, sizeof(double) * 3 * nn));
    TRY(ensure(h->md_im, sizeof(double) * nn));
    if (!s.f) TRY(ensure(h->md_f, sizeof(double) * 3 * nn));
    if (k > 1) TRY(ensure(h->md_fs, sizeof(double) * 3 * nn));
    h->list_on = false;
    TRY(set_batch(h, s.B, s.sys, st));
    EvalIO io;
    io.pos = s.x; io.q = s.q; io.lj = s.lj;
    io.forces = s.f ? s.f : h->md_f.as<double>();      // with k > 1: the fast part during the run
    io.pot = nullptr;
    if (k > 1) { io.fslow = h->md_fs.as<double>(); io.mode = EVAL_SPLIT; }
    TRY(launch_inverse((int)n, s.m, h->md_im.as<double>(), st));
    VVArgs va;
    va.bt = batch_of(h); va.max_units = h->max_units;
    va.x = s.x; va.v = s.v; va.xo = h->md_xo.as<double>();
    va.f = io.forces; va.m = s.m; va.im = h->md_im.as<double>(); va.dt = dt;
    va.fs = nullptr; va.ws = 0.0;
    va.d_oh2 = h->p.d_oh * h->p.d_oh; va.d_hh2 = h->p.d_hh * h->p.d_hh;
    va.tol = shake_tol<T>(); va.tol_v = rattle_tol<T>(); va.max_iter = sizeof(T) == 4 ? 200 : 1000;
    va.status = h->status.as<int>();
    if (s.f && s.f_valid && !h->tune_pending && k == 1) {
        // forces and energies of the start positions come with the systems (whole
        // forces: multiple time stepping needs them split, so it evaluates)
        CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, st));
        for (int b = 0; b < s.B; b++) h->h_e[b] = s.e0[b];
        CUDA_TRY(cudaMemcpy2DAsync(h->sums.p, 4 * sizeof(double), h->h_e, sizeof(double), sizeof(double),
                                   (size_t)s.B, cudaMemcpyHostToDevice, st));
    } else {
        // (also when the autotuner still has to run: it settles the bricks before
        // the lists are sized for them; the forces it recomputes are bitwise the same)
        TRY(evaluate(h, io, s.B, s.sys, st));
    }
    if (h->p.list_skin > 0 && s.B == 1 && n > 0) TRY(list_setup<T>(h, s, !(s.f && s.f_valid), st));
    if (uk) {
        CUDA_TRY(cudaMemsetAsync(h->ctr.p, 0, sizeof(int), st));
        TRY(record_uk(h, s, uk, uk_stride, st));
    }
    h->list_on = h->vl_ctl.p != nullptr && h->p.list_skin > 0 && s.B == 1 && n > 0;
    const bool graphs = (h->p.flags & MSM_FLAG_GRAPHS) && !h->prof.on;
    bool captured = false;
    int rc = MSM_OK;
    const bool warm = graphs && !h->tune_pending && h->gexec &&
                      [&] { const GraphKey k = graph_key(h, s, io, dt, uk, uk_stride);
                            return memcmp(&k, &h->gkey, sizeof k) == 0; }();
    // one md_step is one step, or one outer step of k steps (multiple time stepping)
    for (int step = 0; step < n_steps / k && rc == MSM_OK; step++) {
        if (!graphs || (step == 0 && !warm) || h->tune_pending) {
            rc = md_step<T>(h, s, io, va, uk, uk_stride, st);
            continue;
        }
        if (!captured) {
            rc = md_graph<T>(h, s, io, va, dt, uk, uk_stride);
            captured = true;
        }
        if (rc == MSM_OK) {
            const cudaError_t e = cudaGraphLaunch(h->gexec, st);
            if (e != cudaSuccess) rc = fail_cuda(e, "cudaGraphLaunch", __FILE__, __LINE__);
            else count_launch((int)h->g_kernels);
        }
    }
    h->list_on = false;
    // the caller's forces are the whole forces at the end positions (the last
    // evaluation of an outer step is a split one)
    if (rc == MSM_OK && k > 1 && s.f) rc = launch_add(3 * n, h->md_fs.as<double>(), s.f, st);
    return rc;
}

static int run_md(msm_handle *h, const RunSys &s, double dt, int n_steps, double *uk, int64_t uk_stride,
                  cudaStream_t st)
{
    if (!(dt > 0) || n_steps < 0) return fail_msg(MSM_EINVAL, "dt must be > 0 and n_steps >= 0");
    for (int b = 0; b < s.B; b++)
        if (s.sys[b].n_mol > 0 && h->p.model != MSM_MODEL_WATER)
            return fail_msg(MSM_EINVAL, "rigid molecules need the water model");
    if (h->precision == MSM_FP32) return run_md_t<float>(h, s, dt, n_steps, uk, uk_stride, st);
    return run_md_t<double>(h, s, dt, n_steps, uk, uk_stride, st);
}

static int check_system(const msm_system *sys)
{
    if (!sys) return fail_msg(MSM_EINVAL, "system is NULL");
    if (sys->n < 0 || sys->n_mol < 0 || 3 * sys->n_mol > sys->n) return fail_msg(MSM_EINVAL, "bad atom counts");
    if (sys->n > 0 && (!sys->x || !sys->v || !sys->q || !sys->m)) return fail_msg(MSM_EINVAL, "x, v, q, m are required");
    return MSM_OK;
}

extern "C" int md_run(msm_handle *h, msm_system *sys, double dt, int32_t n_steps, double *uk, void *stream)
{
    if (!h) return fail_msg(MSM_EINVAL, "handle is NULL");
    TRY(check_system(sys));
    TRY(check_arrays({sys->x, sys->v, sys->q, sys->m, sys->lj, sys->f, uk}));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = (size_t)sys->n;
    SysIn si;
    si.n = sys->n; si.n_mol = sys->n_mol;
    memcpy(si.box, sys->box, sizeof si.box);
    RunSys s;
    s.B = 1; s.sys = &si;
    const bool x_host = sys->x && !on_device(sys->x), v_host = sys->v && !on_device(sys->v);
    if (x_host) {
        TRY(ensure(h->md_x, sizeof(double) * 3 * nn));
        CUDA_TRY(cudaMemcpyAsync(h->md_x.p, sys->x, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, st));
        s.x = h->md_x.as<double>();
    } else s.x = sys->x;
    if (v_host) {
        TRY(ensure(h->md_v, sizeof(double) * 3 * nn));
        CUDA_TRY(cudaMemcpyAsync(h->md_v.p, sys->v, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, st));
        s.v = h->md_v.as<double>();
    } else s.v = sys->v;
    const void *dq, *dm, *dl;
    TRY(stage_in(h->md_q, sys->q, sizeof(double) * nn, &dq, st));
    TRY(stage_in(h->md_m, sys->m, sizeof(double) * nn, &dm, st));
    TRY(stage_in(h->md_lj, sys->lj, nn, &dl, st));
    s.q = (const double *)dq; s.m = (const double *)dm; s.lj = (const uint8_t *)dl;
    const bool uk_host = uk && !on_device(uk);
    const size_t ukn = 2 * (size_t)(n_steps + 1);
    if (uk_host) TRY(ensure(h->md_uk, sizeof(double) * ukn));
    double *ukd = uk_host ? h->md_uk.as<double>() : uk;
    const bool f_host = sys->f && !on_device(sys->f);
    double e0 = sys->energy;
    if (sys->f) {
        if (f_host) {
            TRY(ensure(h->out_f, sizeof(double) * 3 * nn));
            if (sys->f_valid)
                CUDA_TRY(cudaMemcpyAsync(h->out_f.p, sys->f, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, st));
            s.f = h->out_f.as<double>();
        } else s.f = sys->f;
        s.f_valid = sys->f_valid != 0;
        s.e0 = &e0;
    }
    TRY(run_md(h, s, dt, n_steps, ukd, (int64_t)ukn, st));
    if (x_host) CUDA_TRY(cudaMemcpyAsync(sys->x, s.x, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (v_host) CUDA_TRY(cudaMemcpyAsync(sys->v, s.v, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (uk_host) CUDA_TRY(cudaMemcpyAsync(uk, ukd, sizeof(double) * ukn, cudaMemcpyDeviceToHost, st));
    if (f_host) CUDA_TRY(cudaMemcpyAsync(sys->f, s.f, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (sys->f) CUDA_TRY(cudaMemcpyAsync(&h->h_scal[5], h->sums.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(finish(h, st));
    if (sys->f) { sys->f_valid = 1; sys->energy = h->h_scal[5]; }
    return MSM_OK;
}

// Gather a batch of caller systems into the handle's concatenated buffers.
static int gather_systems(msm_handle *h, int B, const msm_system *systems, std::vector<SysIn> &sys,
                          std::vector<int64_t> &off, bool need_v, cudaStream_t st)
{
    sys.resize((size_t)B);
    off.assign((size_t)B + 1, 0);
    for (int b = 0; b < B; b++) {
        const msm_system &S = systems[b];
        if (S.n < 0 || S.n_mol < 0 || 3 * S.n_mol > S.n) return fail_msg(MSM_EINVAL, "bad atom counts (system %d)", b);
        if (S.n > 0 && (!S.x || !S.q || (need_v && (!S.v || !S.m))))
            return fail_msg(MSM_EINVAL, "system %d lacks x, v, q or m", b);
        TRY(check_arrays({S.x, S.v, S.q, S.m, S.lj, S.f}));
        sys[(size_t)b].n = S.n; sys[(size_t)b].n_mol = S.n_mol;
        memcpy(sys[(size_t)b].box, S.box, sizeof S.box);
        off[(size_t)b + 1] = off[(size_t)b] + S.n;
    }
    const size_t n = (size_t)off[(size_t)B], nn = n > 0 ? n : 1;
    TRY(ensure(h->md_x, sizeof(double) * 3 * nn));
    TRY(ensure(h->md_q, sizeof(double) * nn));
    TRY(ensure(h->md_lj, nn));
    if (need_v) {
        TRY(ensure(h->md_v, sizeof(double) * 3 * nn));
        TRY(ensure(h->md_m, sizeof(double) * nn));
    }
    for (int b = 0; b < B; b++) {
        const msm_system &S = systems[b];
        const size_t o = (size_t)off[(size_t)b], m = (size_t)S.n;
        if (!m) continue;
        CUDA_TRY(cudaMemcpyAsync(h->md_x.as<double>() + 3 * o, S.x, sizeof(double) * 3 * m, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(h->md_q.as<double>() + o, S.q, sizeof(double) * m, cudaMemcpyDefault, st));
        if (S.lj) CUDA_TRY(cudaMemcpyAsync(h->md_lj.as<uint8_t>() + o, S.lj, m, cudaMemcpyDefault, st));
        else CUDA_TRY(cudaMemsetAsync(h->md_lj.as<uint8_t>() + o, 0, m, st));
        if (need_v) {
            CUDA_TRY(cudaMemcpyAsync(h->md_v.as<double>() + 3 * o, S.v, sizeof(double) * 3 * m, cudaMemcpyDefault, st));
            CUDA_TRY(cudaMemcpyAsync(h->md_m.as<double>() + o, S.m, sizeof(double) * m, cudaMemcpyDefault, st));
        }
    }
    return MSM_OK;
}

extern "C" int msm_system_forces_batched(msm_handle *h, int32_t n_sys, msm_system *systems, double *energies,
                                         void *stream)
{
    if (!h || n_sys < 1 || !systems) return fail_msg(MSM_EINVAL, "bad batched arguments");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<SysIn> sys;
    std::vector<int64_t> off;
    TRY(gather_systems(h, n_sys, systems, sys, off, false, st));
    const size_t n = (size_t)off[(size_t)n_sys];
    TRY(ensure(h->md_f, sizeof(double) * 3 * (n > 0 ? n : 1)));
    EvalIO io;
    io.pos = h->md_x.as<double>(); io.q = h->md_q.as<double>(); io.lj = h->md_lj.as<uint8_t>();
    io.forces = h->md_f.as<double>(); io.pot = nullptr;
    TRY(evaluate(h, io, n_sys, sys.data(), st));
    for (int b = 0; b < n_sys; b++)
        if (systems[b].f && systems[b].n > 0)
            CUDA_TRY(cudaMemcpyAsync(systems[b].f, h->md_f.as<double>() + 3 * off[(size_t)b],
                                     sizeof(double) * 3 * (size_t)systems[b].n, cudaMemcpyDefault, st));
    TRY(copy_sums(h->h_e, h, 0, st));
    TRY(finish(h, st));
    for (int b = 0; b < n_sys; b++) {
        if (energies) energies[b] = h->h_e[b];
        if (systems[b].f) { systems[b].f_valid = 1; systems[b].energy = h->h_e[b]; }
    }
    return MSM_OK;
}

extern "C" int md_run_batched(msm_handle *h, int32_t n_sys, msm_system *systems, double dt, int32_t n_steps,
                              double *uk, void *stream)
{
    if (!h || n_sys < 1 || !systems) return fail_msg(MSM_EINVAL, "bad batched arguments");
    TRY(check_arrays({uk}));
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<SysIn> sys;
    std::vector<int64_t> off;
    TRY(gather_systems(h, n_sys, systems, sys, off, true, st));
    const size_t n = (size_t)off[(size_t)n_sys];
    // forces carried in only when every system brings valid ones
    bool carry = true;
    for (int b = 0; b < n_sys; b++) carry = carry && systems[b].f && systems[b].f_valid;
    bool want_f = false;
    for (int b = 0; b < n_sys; b++) want_f = want_f || systems[b].f;
    TRY(ensure(h->out_f, sizeof(double) * 3 * (n > 0 ? n : 1)));
    std::vector<double> e0((size_t)n_sys, 0.0);
    if (carry)
        for (int b = 0; b < n_sys; b++) {
            e0[(size_t)b] = systems[b].energy;
            if (systems[b].n > 0)
                CUDA_TRY(cudaMemcpyAsync(h->out_f.as<double>() + 3 * off[(size_t)b], systems[b].f,
                                         sizeof(double) * 3 * (size_t)systems[b].n, cudaMemcpyDefault, st));
        }
    RunSys s;
    s.B = n_sys; s.sys = sys.data();
    s.x = h->md_x.as<double>(); s.v = h->md_v.as<double>(); s.q = h->md_q.as<double>(); s.m = h->md_m.as<double>();
    s.lj = h->md_lj.as<uint8_t>();
    s.f = h->out_f.as<double>(); s.f_valid = carry; s.e0 = e0.data();
    const int64_t ukn = 2 * (int64_t)(n_steps + 1);
    const bool uk_host = uk && !on_device(uk);
    if (uk_host) TRY(ensure(h->md_uk, sizeof(double) * (size_t)(ukn * n_sys)));
    double *ukd = uk_host ? h->md_uk.as<double>() : uk;
    TRY(run_md(h, s, dt, n_steps, ukd, ukn, st));
    for (int b = 0; b < n_sys; b++) {
        const size_t o = (size_t)off[(size_t)b], m = (size_t)systems[b].n;
        if (!m) continue;
        CUDA_TRY(cudaMemcpyAsync(systems[b].x, s.x + 3 * o, sizeof(double) * 3 * m, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(systems[b].v, s.v + 3 * o, sizeof(double) * 3 * m, cudaMemcpyDefault, st));
        if (systems[b].f) CUDA_TRY(cudaMemcpyAsync(systems[b].f, s.f + 3 * o, sizeof(double) * 3 * m, cudaMemcpyDefault, st));
    }
    if (uk_host) CUDA_TRY(cudaMemcpyAsync(uk, ukd, sizeof(double) * (size_t)(ukn * n_sys), cudaMemcpyDeviceToHost, st));
    if (want_f) TRY(copy_sums(h->h_e, h, 0, st));
    TRY(finish(h, st));
    for (int b = 0; b < n_sys; b++)
        if (systems[b].f) { systems[b].f_valid = 1; systems[b].energy = h->h_e[b]; }
    return MSM_OK;
}

// -------------------------------------------------------------- profiling

extern "C" int msm_profile_enable(msm_handle *h, int32_t on)
{
    if (!h) return fail_msg(MSM_EINVAL, "handle is NULL");
    h->prof.on = on != 0;
    return MSM_OK;
}

extern "C" int msm_profile_read(msm_handle *h, double *ms, int64_t *launches, int32_t max, int32_t reset)
{
    if (!h) return fail_msg(MSM_EINVAL, "handle is NULL");
    for (int i = 0; i < N_STAGES && i < max; i++) {
        if (ms) ms[i] = h->prof.ms[i];
        if (launches) launches[i] = h->prof.cnt[i];
    }
    if (reset)
        for (int i = 0; i < N_STAGES; i++) { h->prof.ms[i] = 0; h->prof.cnt[i] = 0; }
    return N_STAGES;
}

extern "C" const char *msm_stage_name(int32_t stage)
{
    return (stage >= 0 && stage < N_STAGES) ? kStageNames[stage] : "";
}

// ---------------------------------------------------------- pair counting

template <typename T>
static int count_pairs_t(msm_handle *h, int64_t *out)
{
    cudaStream_t st = 0;
    ShortArgs<T> s = short_args<T>(h);
    s.sr = nullptr; s.lj = nullptr; s.cnt = h->eatom.as<double>();
    CUDA_TRY(cudaMemsetAsync(h->eatom.p, 0, sizeof(double) * (size_t)(h->N > 0 ? h->N : 1), st));
    TRY(launch_count_pairs<T>(s, st));
    const double *cols[1] = {h->eatom.as<double>()};
    TRY(launch_sum(batch_of(h), h->max_n, h->PB, 1, cols, h->partials.as<double>(), h->kin_s.as<double>(), 1,
                   h->status.as<int>(), st));
    TRY(ensure_host_e(h, h->B));
    CUDA_TRY(cudaMemcpyAsync(h->h_e, h->kin_s.p, sizeof(double) * (size_t)h->B, cudaMemcpyDeviceToHost, st));
    TRY(finish(h, st));
    double t = 0;
    for (int b = 0; b < h->B; b++) t += h->h_e[b];
    *out = (int64_t)t;
    return MSM_OK;
}

extern "C" int msm_count_pairs(msm_handle *h, int64_t *ordered_pairs)
{
    if (!h || !h->have_geom || !ordered_pairs) return fail_msg(MSM_EINVAL, "no evaluation yet");
    CUDA_TRY(cudaDeviceSynchronize());
    if (h->precision == MSM_FP32) return count_pairs_t<float>(h, ordered_pairs);
    return count_pairs_t<double>(h, ordered_pairs);
}

// ----------------------------------------------------------------- parareal

// Parareal (Sec. 4) on one GPU.  The fine propagations F of an iteration run
// as one batch (md_run_batched over the slices of the iteration); the
// sequential correction sweep runs the coarse propagations G slice by slice.
// The sweep is enqueued without any host synchronisation: each G's status word
// is folded on the device into the sweep's (first failure, with its slice),
// the per-slice max |dx| and the projection status are read once, after the
// sweep.  The iteration runs over a window of slices [b, e) (Sec. 4's
// computational window):
//   plain   (parareal_run): the window is the whole run, b = the iteration
//           index (slices before it are exact: the bracket G(lambda^{k+1}_n) -
//           G(lambda^k_n) vanishes bitwise, so they are copied, not recomputed),
//           stop when the largest change of an iteration is <= tol;
//   sliding (parareal_run_window): at most W slices; after an iteration b moves
//           past slice b (exact) and the converged slices that follow it
//           (max |dx| <= tol), and new slices enter at the end with the coarse
//           propagation of the last window state as their first iterate; stop
//           when b reaches n_slices.  Device memory holds W + 1 states, not
//           n_slices + 1.
// States live in slot n mod (W + 1) (lambda) and n mod W (G of the current
// iterate); the F batch is gathered into slots 0 .. e-b-1 of its own buffer.
struct PararealRun {
    const msm_params *G, *F;
    double dtG, dtF;
    int stepsG, stepsF;
    const msm_system *s0;
    int n_slices, window, max_iter;
    bool sliding;
    double tol;
    double *slices_x, *slices_v;
    int *iters_done;
    double *last_dx;
    int resume_k = -1;     // plain mode: continue from the iterate lambda^k held in slices_x/v (-1: start)
};

static int parareal_impl(const PararealRun &P, cudaStream_t st)
{
    const msm_system &s0 = *P.s0;
    msm_handle *hG = nullptr, *hF = nullptr;
    TRY(msm_create(P.G, &hG));
    int rc = msm_create(P.F, &hF);
    if (rc) { msm_destroy(hG); return rc; }
    const int ns = P.n_slices, W = P.window;
    const size_t n3 = 3 * (size_t)s0.n, nn = (size_t)s0.n, w = (size_t)W;
    const size_t nblk = (n3 + 255) / 256;
    DevBuf lam_x, lam_v, new_x, new_v, gold_x, gold_v, f_x, f_v, cur_x, cur_v, tmp_x, tmp_v, q, m, lj, part, dxs,
        pst, gst;
    double *h_dx = nullptr;
    int *h_st = nullptr;
    auto cleanup = [&]() {
        DevBuf *all[] = {&lam_x, &lam_v, &new_x, &new_v, &gold_x, &gold_v, &f_x, &f_v, &cur_x, &cur_v, &tmp_x,
                         &tmp_v, &q, &m, &lj, &part, &dxs, &pst, &gst};
        for (DevBuf *b : all) release(*b);
        if (h_dx) cudaFreeHost(h_dx);
        if (h_st) cudaFreeHost(h_st);
        msm_destroy(hG);
        msm_destroy(hF);
    };
    auto body = [&]() -> int {
        TRY(ensure(lam_x, sizeof(double) * n3 * (w + 1)));
        TRY(ensure(lam_v, sizeof(double) * n3 * (w + 1)));
        if (!P.sliding) {
            // plain mode keeps the previous iterate whole until a sweep has succeeded
            // (a diverged sweep hands it back): the sweep writes a second set of states
            TRY(ensure(new_x, sizeof(double) * n3 * (w + 1)));
            TRY(ensure(new_v, sizeof(double) * n3 * (w + 1)));
        }
        TRY(ensure(gold_x, sizeof(double) * n3 * w));
        TRY(ensure(gold_v, sizeof(double) * n3 * w));
        TRY(ensure(f_x, sizeof(double) * n3 * w));
        TRY(ensure(f_v, sizeof(double) * n3 * w));
        TRY(ensure(cur_x, sizeof(double) * n3));
        TRY(ensure(cur_v, sizeof(double) * n3));
        TRY(ensure(tmp_x, sizeof(double) * n3));
        TRY(ensure(tmp_v, sizeof(double) * n3));
        TRY(ensure(q, sizeof(double) * nn * w));            // per-slice copies for the batched F
        TRY(ensure(m, sizeof(double) * nn * w));
        TRY(ensure(lj, nn * w));
        TRY(ensure(part, sizeof(double) * nblk * w));
        TRY(ensure(dxs, sizeof(double) * w));
        TRY(ensure(pst, sizeof(int)));
        TRY(ensure(gst, sizeof(int) * 4));
        CUDA_TRY(cudaMallocHost(&h_dx, sizeof(double) * w));
        CUDA_TRY(cudaMallocHost(&h_st, sizeof(int) * 8));
        CUDA_TRY(cudaMemsetAsync(pst.p, 0, sizeof(int), st));
        // projection of corrected states: threshold 10x, target 1x the fine propagator's SHAKE tolerance
        const double ptol = P.F->precision == MSM_FP32 ? shake_tol<float>() : shake_tol<double>();
        const double d_oh2 = P.F->d_oh * P.F->d_oh, d_hh2 = P.F->d_hh * P.F->d_hh;
        auto LX = [&](int n) { return lam_x.as<double>() + (size_t)(n % (W + 1)) * n3; };
        auto LV = [&](int n) { return lam_v.as<double>() + (size_t)(n % (W + 1)) * n3; };
        // where the sweep writes the new iterate: the same slots (sliding) or the second set (plain)
        auto NXp = [&](int n) { return (P.sliding ? lam_x : new_x).as<double>() + (size_t)(n % (W + 1)) * n3; };
        auto NVp = [&](int n) { return (P.sliding ? lam_v : new_v).as<double>() + (size_t)(n % (W + 1)) * n3; };
        auto GX = [&](int n) { return gold_x.as<double>() + (size_t)(n % W) * n3; };
        auto GV = [&](int n) { return gold_v.as<double>() + (size_t)(n % W) * n3; };
        auto D2D = [&](double *dst, const double *src) {
            return cudaMemcpyAsync(dst, src, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
        };
        CUDA_TRY(cudaMemcpyAsync(LX(0), s0.x, sizeof(double) * n3, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(LV(0), s0.v, sizeof(double) * n3, cudaMemcpyDefault, st));
        for (size_t k = 0; k < w; k++) {
            CUDA_TRY(cudaMemcpyAsync(q.as<double>() + k * nn, s0.q, sizeof(double) * nn, cudaMemcpyDefault, st));
            CUDA_TRY(cudaMemcpyAsync(m.as<double>() + k * nn, s0.m, sizeof(double) * nn, cudaMemcpyDefault, st));
            if (s0.lj) CUDA_TRY(cudaMemcpyAsync(lj.as<uint8_t>() + k * nn, s0.lj, nn, cudaMemcpyDefault, st));
            else CUDA_TRY(cudaMemsetAsync(lj.as<uint8_t>() + k * nn, 0, nn, st));
        }
        // the caller's copy of slice n's end state (slot n+1 of slices_x/v)
        auto publish = [&](int n1) -> int {
            CUDA_TRY(cudaMemcpyAsync(P.slices_x + (size_t)n1 * n3, LX(n1), sizeof(double) * n3, cudaMemcpyDefault, st));
            CUDA_TRY(cudaMemcpyAsync(P.slices_v + (size_t)n1 * n3, LV(n1), sizeof(double) * n3, cudaMemcpyDefault, st));
            return MSM_OK;
        };
        TRY(publish(0));
        SysIn si;
        si.n = s0.n; si.n_mol = s0.n_mol;
        memcpy(si.box, s0.box, sizeof si.box);
        std::vector<SysIn> sis(w, si);
        // G on tmp, no host synchronisation; its status is folded into gst (tag = slice).
        // With Verlet lists G needs the host between runs (list maintenance): it then
        // synchronises after each propagation, as md_run does.
        const bool g_sync = P.G->list_skin > 0;
        auto runG = [&](int slice) -> int {
            RunSys t;
            t.B = 1; t.sys = &si; t.x = tmp_x.as<double>(); t.v = tmp_v.as<double>();
            t.q = q.as<double>(); t.m = m.as<double>(); t.lj = lj.as<uint8_t>();
            int r = run_md(hG, t, P.dtG, P.stepsG, nullptr, 0, st);
            if (r == MSM_OK && g_sync) r = finish(hG, st);
            if (r != MSM_OK) {
                char msg[512];
                snprintf(msg, sizeof msg, "%s", msm_last_error());
                return fail_msg(r, "coarse propagator G: %s", msg);
            }
            return launch_status_fold(hG->status.as<int>(), gst.as<int>(), slice, st);
        };
        // read the sweep's outcome: per-slice changes, first G failure, projection status
        auto read_sweep = [&](int nseg, int *g_status) -> int {
            if (nseg > 0) {
                TRY(launch_max_reduce_seg(nseg, (int)nblk, part.as<double>(), dxs.as<double>(), st));
                CUDA_TRY(cudaMemcpyAsync(h_dx, dxs.p, sizeof(double) * (size_t)nseg, cudaMemcpyDeviceToHost, st));
            }
            CUDA_TRY(cudaMemcpyAsync(h_st, gst.p, sizeof(int) * 4, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaMemcpyAsync(h_st + 4, pst.p, sizeof(int), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            prof_resolve(hG);
            if (h_st[4]) return fail_msg(MSM_ENOCONV, "projection of a corrected slice onto the rigid "
                                                      "constraints did not converge");
            *g_status = h_st[0];
            return MSM_OK;
        };
        auto g_failure = [&](int it) {
            const int code = h_st[0], kind = h_st[1], slice = h_st[2], atom = h_st[3] - 1;
            char what[256];
            if (code == MSM_ENOCONV && kind)
                snprintf(what, sizeof what, "%s did not converge (molecule starting at atom %d)",
                         kind == 1 ? "SHAKE" : "RATTLE", atom);
            else
                snprintf(what, sizeof what, "%s", status_text(code));
            return fail_msg(MSM_ENOCONV, "parareal: diverged at iteration %d, slice %d (coarse propagator G: %s)",
                            it, slice, what);
        };
        // first iterates of slices [e0, e1): lambda^0_{n+1} = G(lambda^0_n), sequentially
        auto fill = [&](int e0, int e1) -> int {
            for (int n = e0; n < e1; n++) {
                CUDA_TRY(D2D(tmp_x.as<double>(), LX(n)));
                CUDA_TRY(D2D(tmp_v.as<double>(), LV(n)));
                TRY(runG(n));
                CUDA_TRY(D2D(GX(n), tmp_x.as<double>()));
                CUDA_TRY(D2D(GV(n), tmp_v.as<double>()));
                CUDA_TRY(D2D(LX(n + 1), tmp_x.as<double>()));
                CUDA_TRY(D2D(LV(n + 1), tmp_v.as<double>()));
            }
            return MSM_OK;
        };
        CUDA_TRY(cudaMemsetAsync(gst.p, 0, sizeof(int) * 4, st));
        int b = 0, e = std::min(W, ns);
        const int k_start = P.resume_k >= 0 ? P.resume_k : 0;
        if (P.resume_k >= 0) {
            // resume: lambda^k_n from the caller (n = 0 .. n_slices), and G(lambda^k_n) of every
            // slice, which the sweep of iteration k-1 left behind -- recomputed by the same
            // propagation on the same states, so the iterates continue bit for bit
            for (int n = 1; n <= ns; n++) {
                CUDA_TRY(cudaMemcpyAsync(LX(n), P.slices_x + (size_t)n * n3, sizeof(double) * n3, cudaMemcpyDefault, st));
                CUDA_TRY(cudaMemcpyAsync(LV(n), P.slices_v + (size_t)n * n3, sizeof(double) * n3, cudaMemcpyDefault, st));
            }
            for (int n = 0; n < ns; n++) {
                CUDA_TRY(D2D(tmp_x.as<double>(), LX(n)));
                CUDA_TRY(D2D(tmp_v.as<double>(), LV(n)));
                TRY(runG(n));
                CUDA_TRY(D2D(GX(n), tmp_x.as<double>()));
                CUDA_TRY(D2D(GV(n), tmp_v.as<double>()));
            }
        } else {
            TRY(fill(0, e));
        }
        int done = k_start;
        double dxh = INFINITY;
        bool diverged = false;
        {
            int gs = 0;
            TRY(read_sweep(0, &gs));
            if (gs) return fail_msg(MSM_ENOCONV, "coarse propagator G failed on the initial sweep (%s)",
                                    status_text(gs));
        }
        if (P.sliding) for (int n = 1; n <= e; n++) TRY(publish(n));
        for (int it = k_start; it < k_start + P.max_iter && b < ns; it++) {
            if (P.sliding) {
                // refill the window: first iterates of the slices entering it, by G in order
                const int e2 = std::min(b + W, ns);
                if (e2 > e) {
                    CUDA_TRY(cudaMemsetAsync(gst.p, 0, sizeof(int) * 4, st));
                    TRY(fill(e, e2));
                    for (int n = e + 1; n <= e2; n++) TRY(publish(n));
                    e = e2;
                    int g2 = 0;
                    TRY(read_sweep(0, &g2));
                    if (g2) { g_failure(it + 1); diverged = true; break; }
                }
            }
            if (!P.sliding) b = std::min(it, ns);              // slices before the iteration index are exact
            if (b >= e) {
                // plain mode, every slice exact: this iteration would change nothing
                done = it + 1;
                dxh = 0;
                break;
            }
            const int nb = e - b;
            // f_n = F(lambda^k_n) for every slice of the window: one batch
            for (int n = b; n < e; n++) {
                CUDA_TRY(D2D(f_x.as<double>() + (size_t)(n - b) * n3, LX(n)));
                CUDA_TRY(D2D(f_v.as<double>() + (size_t)(n - b) * n3, LV(n)));
            }
            {
                RunSys t;
                t.B = nb; t.sys = sis.data(); t.x = f_x.as<double>(); t.v = f_v.as<double>();
                t.q = q.as<double>(); t.m = m.as<double>(); t.lj = lj.as<uint8_t>();
                int r = run_md(hF, t, P.dtF, P.stepsF, nullptr, 0, st);
                if (r == MSM_OK) r = finish(hF, st);
                if (r != MSM_OK) {
                    char msg[512];
                    snprintf(msg, sizeof msg, "%s", msm_last_error());
                    return fail_msg(r, "fine propagator F: %s", msg);
                }
            }
            // sequential correction sweep from the window's first state (final)
            CUDA_TRY(D2D(cur_x.as<double>(), LX(b)));
            CUDA_TRY(D2D(cur_v.as<double>(), LV(b)));
            if (!P.sliding) {                                  // the exact slices carry over unchanged
                CUDA_TRY(cudaMemcpyAsync(NXp(0), LX(0), sizeof(double) * n3 * (size_t)(b + 1), cudaMemcpyDeviceToDevice, st));
                CUDA_TRY(cudaMemcpyAsync(NVp(0), LV(0), sizeof(double) * n3 * (size_t)(b + 1), cudaMemcpyDeviceToDevice, st));
            }
            CUDA_TRY(cudaMemsetAsync(part.p, 0, sizeof(double) * nblk * (size_t)nb, st));
            CUDA_TRY(cudaMemsetAsync(gst.p, 0, sizeof(int) * 4, st));
            for (int n = b; n < e; n++) {
                CUDA_TRY(D2D(tmp_x.as<double>(), cur_x.as<double>()));
                CUDA_TRY(D2D(tmp_v.as<double>(), cur_v.as<double>()));
                TRY(runG(n));
                const double *fx = f_x.as<double>() + (size_t)(n - b) * n3, *fv = f_v.as<double>() + (size_t)(n - b) * n3;
                TRY(launch_parareal_update((int)n3, fx, tmp_x.as<double>(), GX(n), cur_x.as<double>(), nullptr, nullptr, st));
                TRY(launch_parareal_update((int)n3, fv, tmp_v.as<double>(), GV(n), cur_v.as<double>(), nullptr, nullptr, st));
                TRY(launch_pr_project((int)s0.n_mol, cur_x.as<double>(), cur_v.as<double>(), m.as<double>(), d_oh2,
                                      d_hh2, 10.0 * ptol, ptol, 1e-14, pst.as<int>(), st));
                TRY(launch_absdiff_partials((int)n3, cur_x.as<double>(), LX(n + 1),
                                            part.as<double>() + (size_t)(n - b) * nblk, st));
                CUDA_TRY(D2D(GX(n), tmp_x.as<double>()));
                CUDA_TRY(D2D(GV(n), tmp_v.as<double>()));
                CUDA_TRY(D2D(NXp(n + 1), cur_x.as<double>()));
                CUDA_TRY(D2D(NVp(n + 1), cur_v.as<double>()));
            }
            int gs = 0;
            TRY(read_sweep(nb, &gs));
            if (gs) {
                // the coarse propagator broke down on a corrected state: the iteration diverged.
                // The caller gets the last complete iterate: plain mode still holds it in lam;
                // sliding mode published it after the previous iteration.
                g_failure(it + 1);
                diverged = true;
                break;
            }
            if (!P.sliding) { std::swap(lam_x, new_x); std::swap(lam_v, new_v); }
            dxh = 0;
            for (int k = 0; k < nb; k++) dxh = std::max(dxh, h_dx[k]);
            done = it + 1;
            if (P.sliding) {
                int nb2 = b + 1;                                // slice b's end is exact
                while (nb2 < e && h_dx[nb2 - b] <= P.tol) nb2++;
                for (int n = b + 1; n <= e; n++) TRY(publish(n));
                b = nb2;
            } else if (dxh <= P.tol) {
                break;
            }
        }
        if (!P.sliding)
            for (int n = 1; n <= ns; n++) TRY(publish(n));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (P.iters_done) *P.iters_done = done;
        if (P.last_dx) *P.last_dx = dxh;
        if (diverged) return MSM_ENOCONV;                       // message set by g_failure
        if (P.sliding) {
            if (b < ns) return fail_msg(MSM_ENOCONV, "parareal: %d of %d slices converged after %d iterations",
                                        b, ns, done);
            return MSM_OK;
        }
        if (P.max_iter > 0 && !(dxh <= P.tol)) return fail_msg(MSM_ENOCONV, "parareal: max |dx| = %g after %d iterations", dxh, done);
        return MSM_OK;
    };
    rc = body();
    cleanup();
    return rc;
}

static int parareal_args(const msm_params *G, double dtG, int32_t stepsG, const msm_params *F, double dtF,
                         int32_t stepsF, const msm_system *state0, int32_t n_slices, int32_t max_iter, double tol,
                         double *slices_x, double *slices_v)
{
    if (!G || !F || !state0 || !slices_x || !slices_v) return fail_msg(MSM_EINVAL, "NULL argument");
    if (n_slices < 1 || max_iter < 0 || stepsG < 0 || stepsF < 0 || !(tol >= 0))
        return fail_msg(MSM_EINVAL, "bad parareal sizes");
    if (fabs(dtG * stepsG - dtF * stepsF) > 1e-9 * fabs(dtF * stepsF))
        return fail_msg(MSM_EINVAL, "G and F must span the same slice length");
    const msm_system &s0 = *state0;
    if (s0.n <= 0 || !s0.x || !s0.v || !s0.q || !s0.m) return fail_msg(MSM_EINVAL, "state0 incomplete");
    TRY(check_arrays({s0.x, s0.v, s0.q, s0.m, s0.lj, slices_x, slices_v}));
    return MSM_OK;
}

extern "C" int parareal_run(const msm_params *G, double dtG, int32_t stepsG, const msm_params *F, double dtF,
                            int32_t stepsF, const msm_system *state0, int32_t n_slices, int32_t max_iter, double tol,
                            double *slices_x, double *slices_v, int32_t *iters_done, double *last_dx, void *stream)
{
    TRY(parareal_args(G, dtG, stepsG, F, dtF, stepsF, state0, n_slices, max_iter, tol, slices_x, slices_v));
    PararealRun P{G, F, dtG, dtF, stepsG, stepsF, state0, n_slices, n_slices, max_iter, false, tol,
                  slices_x, slices_v, iters_done, last_dx};
    return parareal_impl(P, (cudaStream_t)stream);
}

extern "C" int parareal_resume(const msm_params *G, double dtG, int32_t stepsG, const msm_params *F, double dtF,
                               int32_t stepsF, const msm_system *state0, int32_t n_slices, int32_t iters_before,
                               int32_t max_iter, double tol, double *slices_x, double *slices_v, int32_t *iters_done,
                               double *last_dx, void *stream)
{
    TRY(parareal_args(G, dtG, stepsG, F, dtF, stepsF, state0, n_slices, max_iter, tol, slices_x, slices_v));
    if (iters_before < 0) return fail_msg(MSM_EINVAL, "iters_before must be >= 0");
    PararealRun P{G, F, dtG, dtF, stepsG, stepsF, state0, n_slices, n_slices, max_iter, false, tol,
                  slices_x, slices_v, iters_done, last_dx};
    P.resume_k = iters_before;
    return parareal_impl(P, (cudaStream_t)stream);
}

extern "C" int parareal_run_window(const msm_params *G, double dtG, int32_t stepsG, const msm_params *F,
                                   double dtF, int32_t stepsF, const msm_system *state0, int32_t n_slices,
                                   int32_t window, int32_t max_iter, double tol, double *slices_x, double *slices_v,
                                   int32_t *iters_done, double *last_dx, void *stream)
{
    TRY(parareal_args(G, dtG, stepsG, F, dtF, stepsF, state0, n_slices, max_iter, tol, slices_x, slices_v));
    if (window < 1) return fail_msg(MSM_EINVAL, "window must be >= 1");
    PararealRun P{G, F, dtG, dtF, stepsG, stepsF, state0, n_slices, std::min(window, n_slices), max_iter, true, tol,
                  slices_x, slices_v, iters_done, last_dx};
    return parareal_impl(P, (cudaStream_t)stream);
}

// -------------------------------------------------------------- inspection

extern "C" int msm_grid_shape(msm_handle *h, int32_t level, int64_t shape[3], int64_t lo[3])
{
    if (!h || !h->have_geom) return fail_msg(MSM_EINVAL, "no evaluation yet");
    if (!has_grids(h->p)) return fail_msg(MSM_EINVAL, "the cutoff methods have no grids");
    if (level < 0 || level >= h->gg.levels) return fail_msg(MSM_EINVAL, "level out of range");
    for (int d = 0; d < 3; d++) {
        if (shape) shape[d] = d ? h->gg.L[level].n[d] : h->gg.L[level].nx_log;
        if (lo) lo[d] = h->gg.L[level].lo[d];
    }
    return MSM_OK;
}

extern "C" int msm_stage_grid(msm_handle *h, int32_t level, int32_t which, double *out, int64_t count)
{
    if (!h || !h->have_geom || !out) return fail_msg(MSM_EINVAL, "no evaluation yet");
    if (!has_grids(h->p)) return fail_msg(MSM_EINVAL, "the cutoff methods have no grids");
    const int l = h->gg.levels;
    if (level < 0 || level >= l || which < 0 || which > 2 || (which == 1 && level == l - 1))
        return fail_msg(MSM_EINVAL, "no such grid");
    const LevelGeom &L = h->gg.L[level];
    // the method's points: nx_log of every stored row of n[0]
    const int64_t rows = (int64_t)L.n[1] * L.n[2], m = (int64_t)L.nx_log * rows;
    if (count < m) return fail_msg(MSM_EINVAL, "output too small");
    CUDA_TRY(cudaDeviceSynchronize());
    if (which == 2 && level == l - 1) {
        CUDA_TRY(cudaMemcpy2D(out, sizeof(double) * L.nx_log, h->utop.p, sizeof(double) * L.n[0],
                              sizeof(double) * L.nx_log, (size_t)rows, cudaMemcpyDeviceToHost));
        return MSM_OK;
    }
    const DevBuf &b = which == 0 ? h->qgrid : (which == 1 ? h->ucut : h->ugrid);
    if (h->precision == MSM_FP64) {
        CUDA_TRY(cudaMemcpy2D(out, sizeof(double) * L.nx_log, b.as<double>() + L.off, sizeof(double) * L.n[0],
                              sizeof(double) * L.nx_log, (size_t)rows, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp((size_t)m);
        CUDA_TRY(cudaMemcpy2D(tmp.data(), sizeof(float) * L.nx_log, b.as<float>() + L.off, sizeof(float) * L.n[0],
                              sizeof(float) * L.nx_log, (size_t)rows, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < m; i++) out[i] = tmp[(size_t)i];
    }
    return MSM_OK;
}

extern "C" int msm_cell_list(msm_handle *h, int64_t *perm, int64_t *cell_start, int64_t *ncells)
{
    if (!h || !h->have_geom) return fail_msg(MSM_EINVAL, "no evaluation yet");
    CUDA_TRY(cudaDeviceSynchronize());
    const int64_t n = h->last_n, nc = h->cg.ncells;
    if (ncells) *ncells = nc;
    if (perm && n > 0) {
        std::vector<int> t((size_t)n);
        CUDA_TRY(cudaMemcpy(t.data(), h->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i < n; i++) perm[i] = t[(size_t)i];
    }
    if (cell_start) {
        std::vector<int> t((size_t)nc + 1);
        CUDA_TRY(cudaMemcpy(t.data(), h->start.p, sizeof(int) * (nc + 1), cudaMemcpyDeviceToHost));
        for (int64_t i = 0; i <= nc; i++) cell_start[i] = t[(size_t)i];
    }
    return MSM_OK;
}

extern "C" int msm_stage_atoms(msm_handle *h, int32_t which, double *out, int64_t count)
{
    if (!h || !h->have_geom || !out) return fail_msg(MSM_EINVAL, "no evaluation yet");
    const int64_t n = h->last_n;
    if (which < 0 || which > 1 || count < (which ? 3 * n : n)) return fail_msg(MSM_EINVAL, "bad stage request");
    CUDA_TRY(cudaDeviceSynchronize());
    std::vector<int> perm((size_t)n);
    std::vector<double> sr((size_t)n * 4);
    CUDA_TRY(cudaMemcpy(perm.data(), h->perm.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
    if (h->precision == MSM_FP64) {
        CUDA_TRY(cudaMemcpy(sr.data(), h->sr.p, sizeof(double) * 4 * n, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> t((size_t)n * 4);
        CUDA_TRY(cudaMemcpy(t.data(), h->sr.p, sizeof(float) * 4 * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < t.size(); i++) sr[i] = t[i];
    }
    for (int64_t i = 0; i < n; i++) {                      // stored by atom index
        if (which == 0) out[i] = sr[4 * i + 3];
        else for (int d = 0; d < 3; d++) out[3 * i + d] = sr[4 * i + d];
    }
    return MSM_OK;
}

extern "C" int msm_list_stats(msm_handle *h, int64_t *out, int32_t max)
{
    if (!h || !out) return fail_msg(MSM_EINVAL, "NULL argument");
    const int64_t v[8] = {h->vl_builds, h->vl_overflows, h->vl_cap, h->vl_cap_lj, VL_ROWS,
                          h->vl_seen[0], h->vl_seen[1], h->vl_seen[2]};
    for (int k = 0; k < 8 && k < max; k++) out[k] = v[k];
    return MSM_OK;
}

extern "C" int msm_diag_convert(int64_t n, const double *x, float *x32, const float *y, double *y64, void *stream)
{
    if (n < 0) return fail_msg(MSM_EINVAL, "n < 0");
    if (n == 0) return MSM_OK;
    if (!on_device(x) || !on_device(x32) || !on_device(y) || !on_device(y64))
        return fail_msg(MSM_EINVAL, "msm_diag_convert takes device arrays");
    cudaStream_t st = (cudaStream_t)stream;
    TRY(launch_diag_convert(n, x, x32, y, y64, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return MSM_OK;
}

extern "C" int64_t msm_kernel_launches(void) { return g_launches.load(); }

extern "C" const char *msm_last_error(void) { return g_err; }
