// msm_api.cu -- the C ABI of libmsm_gb300.so (declared in include/msm.h):
// handle and scratch management, geometry and table set-up, and the
// orchestration of one MSM evaluation (Sec. 3, worked example steps 1-9),
// of velocity Verlet (Sec. 2) and of parareal (Sec. 4).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "kernels.cuh"

using namespace msm;

// ------------------------------------------------------------------ errors

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

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

static int ensure(DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.cap >= bytes) return MSM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return fail_msg(MSM_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    }
    b.cap = bytes;
    return MSM_OK;
}

static void release(DevBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

static bool on_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------------ handle

// Stages timed by the profiler (CUDA events around each stage's launches).
enum Stage { ST_BIN, ST_SHORT, ST_ANTERP, ST_RESTRICT, ST_STENCIL, ST_TOP, ST_PROLONG, ST_INTERP, ST_SUMS,
             ST_VV1, ST_VV2, ST_LIST, N_STAGES };
static const char *kStageNames[N_STAGES] = {"bin_sort",      "short_range", "anterpolation",
                                            "restriction",   "lattice_cutoff", "top_level",
                                            "prolongation",  "interpolation", "exclusions_sums",
                                            "vv_first_shake", "vv_second_rattle", "verlet_list_maintenance"};

struct Profiler {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    size_t used = 0;
    std::vector<int3> marks;        // (stage, begin event, end event)
    double ms[N_STAGES] = {0};
    long long cnt[N_STAGES] = {0};
};

struct msm_handle {
    msm_params p;
    Profiler prof;
    int precision;
    // geometry of the current box
    bool have_geom = false;
    double box[6] = {0, 0, 0, 0, 0, 0};
    CellGeom cg;
    GridGeom gg;
    double inv_h = 0;
    int bd[3] = {4, 2, 2}, nb[3] = {0, 0, 0}, nbricks = 0;
    int64_t last_n = 0;
    // tables
    bool stencil_ready = false;
    StencilGeom sg;
    bool top_ready = false;
    int top_n[3] = {0, 0, 0};
    // scratch
    DevBuf key, count, start, perm, bsum, rel, frac, apos, afrac, akey, aflag, sr, lj;
    DevBuf qgrid, ucut, ugrid, utop, ttop, wst_d, wst_t, rows;
    DevBuf eatom, vatom, kin, partials, sums, status;
    DevBuf in_pos, in_q, in_lj, out_f, out_p;          // staging of host arrays
    DevBuf md_f, md_xo, md_x, md_v, md_q, md_m, md_lj, md_uk, md_im;
    int *h_status = nullptr;
    double *h_scal = nullptr;
    // Verlet lists (md_run with list_skin > 0)
    bool list_on = false;
    DevBuf vl_perm, vl_start, vl_xref, vl_pos, grp_rows, grp_nrows, grp_j, vl_cnt, vl_cntlj, vl_nbr, vl_ctl;
    int vl_cap = 0, vl_jcap = 0, vl_rows = 0, vl_ngroups = 0;
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
    p->lj_sigma = 0.315061;
    p->lj_epsilon = 0.6364;
    p->d_oh = 0.09572;
    p->d_hh = 2.0 * 0.09572 * sin(104.52 * M_PI / 360.0);
    p->wall_k = 0.0;
    p->wall_width = 0.0;
    p->list_skin = 0.0;
}

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
    if (!(p->wall_k >= 0) || !(p->wall_width >= 0)) return fail_msg(MSM_EINVAL, "wall_k and wall_width must be >= 0");
    if (!(p->list_skin >= 0) || !(p->list_skin < p->a)) return fail_msg(MSM_EINVAL, "list_skin must be in [0, a)");
    int rad = 0;
    while ((double)(rad + 1) * p->h < 2.0 * p->a) rad++;
    if (rad > 12) return fail_msg(MSM_EINVAL, "2a/h = %.3g is too large (lattice-cutoff radius %d > 12)", 2 * p->a / p->h, rad);
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
                     &h->akey, &h->aflag, &h->sr, &h->lj, &h->qgrid, &h->ucut, &h->ugrid, &h->utop, &h->ttop,
                     &h->wst_d, &h->wst_t, &h->rows, &h->eatom, &h->vatom, &h->kin, &h->partials, &h->sums,
                     &h->status, &h->in_pos, &h->in_q, &h->in_lj, &h->out_f, &h->out_p, &h->md_f, &h->md_xo,
                     &h->md_x, &h->md_v, &h->md_q, &h->md_m, &h->md_lj, &h->md_uk, &h->md_im,
                     &h->vl_perm, &h->vl_start, &h->vl_xref, &h->vl_pos, &h->grp_rows, &h->grp_nrows,
                     &h->grp_j, &h->vl_cnt, &h->vl_cntlj, &h->vl_nbr, &h->vl_ctl};
    for (DevBuf *b : all) release(*b);
    for (cudaEvent_t e : h->prof.ev) cudaEventDestroy(e);
    if (h->h_status) cudaFreeHost(h->h_status);
    if (h->h_scal) cudaFreeHost(h->h_scal);
    if (h->h_ctl) cudaFreeHost(h->h_ctl);
    delete h;
}

static int64_t floordiv64(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) q--;
    return q;
}

// Grid extents per level (open boundaries): level 0 spans [-1, floor(L/h)+2];
// level k+1 spans [ceil((lo-3)/2), floor((hi+3)/2)], every point with a
// non-zero restriction weight from level k.
static int set_geometry(msm_handle *h, const double box[6], cudaStream_t st)
{
    for (int d = 0; d < 6; d++)
        if (!std::isfinite(box[d])) return fail_msg(MSM_EINVAL, "box has a non-finite entry");
    for (int d = 0; d < 3; d++)
        if (!(box[3 + d] > 0)) return fail_msg(MSM_EINVAL, "box lengths must be positive");
    if (h->have_geom && memcmp(box, h->box, sizeof(double) * 6) == 0) return MSM_OK;
    const double hh = h->p.h;
    CellGeom cg;
    int64_t ncells = 1;
    for (int d = 0; d < 3; d++) {
        cg.origin[d] = box[d];
        double nc = floor(box[3 + d] / hh) + 1.0;
        if (nc > 4.0e6) return fail_msg(MSM_EINVAL, "box too large for h");
        cg.nc[d] = (int)nc;
        ncells *= cg.nc[d];
    }
    if (ncells > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "too many cells (%lld)", (long long)ncells);
    cg.h = hh;
    cg.ncells = (int)ncells;
    GridGeom gg;
    gg.levels = h->p.n_levels;
    int64_t lo[3], hi[3], tot = 0;
    for (int d = 0; d < 3; d++) { lo[d] = -1; hi[d] = (int64_t)floor(box[3 + d] / hh) + 2; }
    for (int k = 0; k < gg.levels; k++) {
        if (k > 0)
            for (int d = 0; d < 3; d++) { lo[d] = -floordiv64(-(lo[d] - 3), 2); hi[d] = floordiv64(hi[d] + 3, 2); }
        int64_t sz = 1;
        for (int d = 0; d < 3; d++) { gg.L[k].lo[d] = (int)lo[d]; gg.L[k].n[d] = (int)(hi[d] - lo[d] + 1); sz *= gg.L[k].n[d]; }
        gg.L[k].off = (int)tot;
        tot += sz;
    }
    if (tot > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "grids too large");
    gg.total = (int)tot;
    h->cg = cg;
    h->gg = gg;
    h->inv_h = 1.0 / hh;
    memcpy(h->box, box, sizeof(double) * 6);
    h->have_geom = true;

    const size_t ts = h->precision == MSM_FP32 ? sizeof(float) : sizeof(double);
    TRY(ensure(h->count, sizeof(int) * (size_t)(ncells + 1)));
    TRY(ensure(h->start, sizeof(int) * (size_t)(ncells + 1)));
    TRY(ensure(h->bsum, sizeof(int) * (size_t)scan_scratch_ints()));
    TRY(ensure(h->qgrid, ts * (size_t)tot));
    TRY(ensure(h->ucut, ts * (size_t)tot));
    TRY(ensure(h->ugrid, ts * (size_t)tot));
    const LevelGeom &top = gg.L[gg.levels - 1];
    TRY(ensure(h->utop, sizeof(double) * (size_t)top.n[0] * top.n[1] * top.n[2]));
    // top-level Toeplitz table g^{l-1} over all offsets (FP64), rebuilt when its extent changes
    if (!h->top_ready || memcmp(h->top_n, top.n, sizeof h->top_n) != 0) {
        const size_t m = (size_t)(2 * top.n[0] - 1) * (2 * top.n[1] - 1) * (2 * top.n[2] - 1);
        TRY(ensure(h->ttop, sizeof(double) * m));
        const double sc = ldexp(1.0, gg.levels - 1);
        TRY(launch_top_table(top, sc * h->p.a, sc * hh, h->ttop.as<double>(), st));
        memcpy(h->top_n, top.n, sizeof h->top_n);
        h->top_ready = true;
    }
    // lattice-cutoff weights W[n] = g^0(|n| h), |n| h < 2a, and the rows of the tap sphere
    if (!h->stencil_ready) {
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
    return MSM_OK;
}

// Brick shape for the short-range kernel: about 24 atoms per warp at the
// system's mean density (one i atom per lane).
static void choose_bricks(msm_handle *h, int64_t n)
{
    static const int shapes[7][3] = {{1, 1, 1}, {2, 1, 1}, {2, 2, 1}, {2, 2, 2}, {4, 2, 2}, {4, 4, 2}, {4, 4, 4}};
    const double per_cell = (double)n / (double)h->cg.ncells;
    int pick = 0;
    for (int s = 0; s < 7; s++) {
        const int vol = shapes[s][0] * shapes[s][1] * shapes[s][2];
        if (per_cell * vol <= 24.0) pick = s;
    }
    for (int d = 0; d < 3; d++) {
        h->bd[d] = shapes[pick][d];
        h->nb[d] = (h->cg.nc[d] + h->bd[d] - 1) / h->bd[d];
    }
    h->nbricks = h->nb[0] * h->nb[1] * h->nb[2];
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
    TRY(ensure(h->sr, 4 * ts * nn));
    TRY(ensure(h->eatom, sizeof(double) * nn));
    TRY(ensure(h->vatom, sizeof(double) * nn));
    TRY(ensure(h->kin, sizeof(double) * nn));
    TRY(ensure(h->partials, sizeof(double) * 4 * (size_t)sum_partials_needed((int)nn)));
    TRY(ensure(h->sums, sizeof(double) * 8));
    TRY(ensure(h->status, sizeof(int) * 4));
    return MSM_OK;
}

// One evaluation on device arrays.  eatom/vatom get per-atom energy and
// virial; sums[0] = U, sums[1] = virial.  No host synchronisation.
struct EvalIO {
    int64_t n;
    const double *pos, *q;
    const uint8_t *lj;       // nullable (device)
    int64_t n_mol;           // rigid triples for the exclusions (model 1)
    double *forces, *pot;    // device, nullable
};

template <typename T>
static int evaluate_t(msm_handle *h, const EvalIO &io, cudaStream_t st)
{
    const int n = (int)io.n;
    int *status = h->status.as<int>();
    const bool model = h->p.model == MSM_MODEL_WATER;
    if (model) TRY(ensure(h->lj, sizeof(vec4<T>) * (size_t)(n > 0 ? n : 1)));

    BinArgs<T> b;
    b.n = n; b.pos = io.pos; b.q = io.q; b.lj = io.lj; b.g = h->cg; b.inv_h = h->inv_h;
    b.key = h->key.as<int>(); b.count = h->count.as<int>(); b.start = h->start.as<int>(); b.perm = h->perm.as<int>();
    b.bsum = h->bsum.as<int>(); b.rel = h->rel.as<vec4<T>>(); b.frac = h->frac.as<vec4<T>>();
    b.apos = h->apos.as<vec4<T>>(); b.afrac = h->afrac.as<vec4<T>>(); b.akey = h->akey.as<int>();
    b.aflag = h->aflag.as<int>(); b.n_mol = model ? (int)io.n_mol : 0; b.status = status;
    { PROF(ST_BIN); TRY(launch_bin<T>(b, st)); }

    // step 1: short range
    ShortArgs<T> s;
    s.g = h->cg;
    for (int d = 0; d < 3; d++) { s.bd[d] = h->bd[d]; s.nb[d] = h->nb[d]; }
    s.nbricks = h->nbricks;
    s.start = h->start.as<int>(); s.apos = h->apos.as<vec4<T>>(); s.aflag = h->aflag.as<int>();
    const double a = h->p.a;
    s.a = (T)a; s.a2 = (T)(a * a); s.a_sel = (T)(a + 1e-3 * h->p.h);
    s.c0 = (T)(GAMMA_C0 / a); s.c1 = (T)(GAMMA_C1 / (a * a * a)); s.c2 = (T)(GAMMA_C2 / (a * a * a * a * a));
    s.d0 = (T)(-2.5 / (a * a * a)); s.d1 = (T)(1.5 / (a * a * a * a * a));
    const double sg2 = h->p.lj_sigma * h->p.lj_sigma;
    const double sa6 = pow(sg2 / (a * a), 3.0);
    s.lj_s2 = (T)sg2; s.lj_4eps = (T)(4.0 * h->p.lj_epsilon); s.lj_24eps = (T)(24.0 * h->p.lj_epsilon);
    s.lj_shift = (T)(4.0 * h->p.lj_epsilon * (sa6 * sa6 - sa6));
    s.perm = h->perm.as<int>();
    s.sr = h->sr.as<vec4<T>>(); s.lj = model ? h->lj.as<vec4<T>>() : nullptr; s.cnt = nullptr; s.status = status;
    s.vl_ctl = h->list_on ? h->vl_ctl.as<int>() : nullptr;
    {
        ListArgs<T> la;
        if (h->list_on) {
            la.g = h->cg;
            for (int d = 0; d < 3; d++) { la.bd[d] = h->bd[d]; la.nb[d] = h->nb[d]; }
            la.ng[0] = h->nb[0]; la.ng[1] = (h->nb[1] + 1) / 2; la.ng[2] = (h->nb[2] + 1) / 2;
            la.ngroups = h->vl_ngroups;
            la.max_rows = h->vl_rows; la.jcap = h->vl_jcap; la.cap = h->vl_cap;
            const double rl = a + h->p.list_skin;
            la.a2 = s.a2; la.rl2 = (T)(rl * rl); la.rl_sel = (T)(rl + 1e-3 * h->p.h);
            la.skin_half2 = (T)(0.25 * h->p.list_skin * h->p.list_skin);
            la.c0 = s.c0; la.c1 = s.c1; la.c2 = s.c2; la.d0 = s.d0; la.d1 = s.d1;
            la.lj_s2 = s.lj_s2; la.lj_4eps = s.lj_4eps; la.lj_24eps = s.lj_24eps; la.lj_shift = s.lj_shift;
            la.model = model; la.n = n; la.x = io.pos; la.q = io.q;
            la.perm = h->perm.as<int>(); la.start = h->start.as<int>(); la.apos = h->apos.as<vec4<T>>();
            la.aflag = h->aflag.as<int>();
            la.vl_perm = h->vl_perm.as<int>(); la.vl_start = h->vl_start.as<int>(); la.vl_xref = h->vl_xref.as<double>();
            la.vl_pos = h->vl_pos.as<vec4<T>>(); la.grp_rows = h->grp_rows.as<int2>();
            la.grp_nrows = h->grp_nrows.as<int>(); la.grp_j = h->grp_j.as<int>();
            la.cnt = h->vl_cnt.as<int>(); la.cntlj = h->vl_cntlj.as<int>(); la.nbr = h->vl_nbr.as<uint16_t>();
            la.ctl = h->vl_ctl.as<int>(); la.sr = s.sr; la.lj = s.lj; la.status = status;
            PROF(ST_LIST);
            TRY(launch_list_maintain<T>(la, st));
        }
        PROF(ST_SHORT);
        if (h->list_on) TRY(launch_list_force<T>(la, st));
        TRY(launch_short<T>(s, model, st));
    }

    // step 2: anterpolation
    T *qg = h->qgrid.as<T>(), *uc = h->ucut.as<T>(), *ug = h->ugrid.as<T>();
    AnterpArgs<T> an;
    an.cg = h->cg; an.L0 = h->gg.L[0]; an.start = h->start.as<int>(); an.afrac = h->afrac.as<vec4<T>>();
    an.q0 = qg; an.status = status;
    { PROF(ST_ANTERP); TRY(launch_anterp<T>(an, st)); }

    // steps 3-4: restriction down the levels, then the lattice cutoff of levels 0..l-2 in one launch
    const int l = h->gg.levels;
    {
        PROF(ST_RESTRICT);
        for (int k = 0; k + 1 < l; k++) TRY(launch_restrict<T>(h->gg.L[k], h->gg.L[k + 1], qg, qg, status, st));
    }
    if (l > 1) {
        StencilArgs<T> sa;
        sa.gg = h->gg; sa.nlev = l - 1; sa.sg = h->sg;
        sa.blk_off[0] = 0;
        for (int k = 0; k < l - 1; k++) {
            stencil_tiles(h->gg.L[k], sa.tiles[k]);
            sa.blk_off[k + 1] = sa.blk_off[k] + sa.tiles[k][0] * sa.tiles[k][1] * sa.tiles[k][2];
        }
        sa.w = h->wst_t.as<T>(); sa.rows = h->rows.as<int4>(); sa.q = qg; sa.ucut = uc; sa.status = status;
        PROF(ST_STENCIL);
        TRY(launch_stencil<T>(sa, h->status.as<int>() + 2, st));
    }
    // step 5: top level in FP64
    const LevelGeom &top = h->gg.L[l - 1];
    { PROF(ST_TOP); TRY(launch_top<T>(top, h->ttop.as<double>(), qg, h->utop.as<double>(), status, st)); }
    // steps 6-7: prolongation back to level 0
    {
        PROF(ST_PROLONG);
        if (l == 1) {
            const int m = top.n[0] * top.n[1] * top.n[2];
            if (sizeof(T) == sizeof(float)) TRY(launch_cast_f64(m, h->utop.as<double>(), reinterpret_cast<float *>(ug), st));
            else CUDA_TRY(cudaMemcpyAsync(ug, h->utop.p, sizeof(double) * m, cudaMemcpyDeviceToDevice, st));
        } else {
            TRY((launch_prolong<T, double>(h->gg.L[l - 2], top, uc, h->utop.as<double>(), ug, status, st)));
            for (int k = l - 3; k >= 0; k--)
                TRY((launch_prolong<T, T>(h->gg.L[k], h->gg.L[k + 1], uc, ug + h->gg.L[k + 1].off, ug, status, st)));
        }
    }
    // step 8-9: interpolation, totals, scatter to the caller's order
    InterpArgs<T> ia;
    ia.n = n; ia.cg = h->cg; ia.L0 = h->gg.L[0]; ia.perm = h->perm.as<int>(); ia.akey = h->akey.as<int>();
    ia.afrac = h->afrac.as<vec4<T>>(); ia.sr = h->sr.as<vec4<T>>(); ia.lj = model ? h->lj.as<vec4<T>>() : nullptr;
    ia.u0 = ug; ia.pos = io.pos; ia.q = io.q; ia.ke = h->p.coulomb_k; ia.self = GAMMA_C0 / a; ia.inv_h = h->inv_h;
    for (int d = 0; d < 3; d++) { ia.box_lo[d] = h->box[d]; ia.box_hi[d] = h->box[d] + h->box[3 + d]; }
    ia.wall_k = model ? h->p.wall_k : 0.0; ia.wall_w = h->p.wall_width;
    ia.forces = io.forces; ia.pot = io.pot; ia.eatom = h->eatom.as<double>(); ia.vatom = h->vatom.as<double>();
    ia.status = status;
    { PROF(ST_INTERP); TRY(launch_interp<T>(ia, st)); }
    PROF(ST_SUMS);
    if (h->p.model == MSM_MODEL_WATER && io.n_mol > 0) {
        ExclArgs ex;
        ex.n_mol = (int)io.n_mol; ex.x = io.pos; ex.q = io.q; ex.ke = h->p.coulomb_k; ex.a = h->p.a;
        ex.forces = io.forces; ex.pot = io.pot; ex.eatom = h->eatom.as<double>(); ex.vatom = h->vatom.as<double>();
        ex.status = status;
        TRY(launch_exclusions<T>(ex, st));
    }
    const double *cols[2] = {h->eatom.as<double>(), h->vatom.as<double>()};
    TRY(launch_sum(n, 2, cols, h->partials.as<double>(), h->sums.as<double>(), status, st));
    return MSM_OK;
}

static int evaluate(msm_handle *h, const EvalIO &io, const double box[6], cudaStream_t st)
{
    if (io.n < 0 || io.n > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "atom count %lld out of range", (long long)io.n);
    if (h->p.model == MSM_MODEL_WATER && (io.n_mol < 0 || 3 * io.n_mol > io.n))
        return fail_msg(MSM_EINVAL, "n_mol inconsistent with n");
    TRY(set_geometry(h, box, st));
    TRY(ensure_atoms(h, io.n));
    choose_bricks(h, io.n);            // follows every change of n or of the box
    h->last_n = io.n;
    CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, st));
    if (h->precision == MSM_FP32) return evaluate_t<float>(h, io, st);
    return evaluate_t<double>(h, io, st);
}

static int list_grow(msm_handle *h, cudaStream_t st);

// Copy the device status word to the host, synchronise, translate.
static int finish(msm_handle *h, cudaStream_t st)
{
    CUDA_TRY(cudaMemcpyAsync(h->h_status, h->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
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

static int copy_scalar(double *dst, const double *dev_src, cudaStream_t st)
{
    if (!dst) return MSM_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, dev_src, sizeof(double), cudaMemcpyDefault, st));
    return MSM_OK;
}

static int forces_impl(msm_handle *h, int64_t n, int64_t n_mol, const double *pos, const double *q,
                       const uint8_t *lj, const double box[6], double *energy, double *forces, double *pot,
                       double *virial, cudaStream_t st)
{
    if (!h) return fail_msg(MSM_EINVAL, "handle is NULL");
    if (!box) return fail_msg(MSM_EINVAL, "box is NULL");
    if (n < 0) return fail_msg(MSM_EINVAL, "n < 0");
    if (n > 0 && (!pos || !q)) return fail_msg(MSM_EINVAL, "pos and q are required");
    const size_t nn = (size_t)n;
    EvalIO io;
    io.n = n; io.n_mol = n_mol;
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
    TRY(evaluate(h, io, box, st));
    if (f_host && n > 0) CUDA_TRY(cudaMemcpyAsync(forces, h->out_f.p, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (p_host && n > 0) CUDA_TRY(cudaMemcpyAsync(pot, h->out_p.p, sizeof(double) * nn, cudaMemcpyDeviceToHost, st));
    TRY(copy_scalar(energy, h->sums.as<double>(), st));
    TRY(copy_scalar(virial, h->sums.as<double>() + 1, st));
    return finish(h, st);
}

extern "C" int msm_energy_forces(msm_handle *h, int64_t n, const double *pos, const double *q, const double box[6],
                                 double *energy, double *forces, double *potentials, double *virial, void *stream)
{
    if (h && h->p.model != MSM_MODEL_CHARGES)
        return fail_msg(MSM_EINVAL, "msm_energy_forces evaluates point charges; use msm_system_forces for the water model");
    return forces_impl(h, n, 0, pos, q, nullptr, box, energy, forces, potentials, virial, (cudaStream_t)stream);
}

extern "C" int msm_system_forces(msm_handle *h, const msm_system *sys, double *energy, double *forces,
                                 double *potentials, void *stream)
{
    if (!sys) return fail_msg(MSM_EINVAL, "system is NULL");
    return forces_impl(h, sys->n, sys->n_mol, sys->x, sys->q, sys->lj, sys->box, energy, forces, potentials,
                       nullptr, (cudaStream_t)stream);
}

extern "C" int msm_energy_forces_batched(msm_handle *h, int32_t n_sys, const int64_t *offsets, const double *pos,
                                         const double *q, const double *boxes, double *energies, double *forces,
                                         double *potentials, void *stream)
{
    if (!h || n_sys < 0 || (n_sys > 0 && (!offsets || !boxes))) return fail_msg(MSM_EINVAL, "bad batched arguments");
    if (h->p.model != MSM_MODEL_CHARGES) return fail_msg(MSM_EINVAL, "batched evaluation takes point charges");
    cudaStream_t st = (cudaStream_t)stream;
    const bool e_dev = energies && on_device(energies);
    for (int s = 0; s < n_sys; s++) {
        const int64_t o = offsets[s], m = offsets[s + 1] - offsets[s];
        if (o < 0 || m < 0) return fail_msg(MSM_EINVAL, "offsets must be non-decreasing from 0");
        double *e = energies ? (e_dev ? energies + s : &h->h_scal[2]) : nullptr;
        TRY(forces_impl(h, m, 0, pos + 3 * o, q + o, nullptr, boxes + 6 * s, e, forces ? forces + 3 * o : nullptr,
                        potentials ? potentials + o : nullptr, nullptr, st));
        if (energies && !e_dev) energies[s] = h->h_scal[2];
    }
    return MSM_OK;
}

// ----------------------------------------------------------------- dynamics

struct SysDev {
    int64_t n, n_mol;
    double *x, *v;
    const double *q, *m;
    const uint8_t *lj;
    double box[6];
    double *f = nullptr;     // device forces carried in/out (nullable)
    int f_valid = 0;
    double energy = 0;
};

// ------------------------------------------------------------ Verlet lists

static int list_alloc(msm_handle *h, int64_t n, size_t vsz)
{
    const size_t nn = (size_t)(n > 0 ? n : 1);
    TRY(ensure(h->vl_perm, sizeof(int) * nn));
    TRY(ensure(h->vl_start, sizeof(int) * ((size_t)h->cg.ncells + 1)));
    TRY(ensure(h->vl_xref, sizeof(double) * 3 * nn));
    TRY(ensure(h->vl_pos, vsz * nn));
    TRY(ensure(h->grp_rows, sizeof(int2) * (size_t)h->vl_ngroups * h->vl_rows));
    TRY(ensure(h->grp_nrows, sizeof(int) * (size_t)h->vl_ngroups));
    TRY(ensure(h->grp_j, sizeof(int) * (size_t)h->vl_ngroups));
    TRY(ensure(h->vl_cnt, sizeof(int) * nn));
    TRY(ensure(h->vl_cntlj, sizeof(int) * nn));
    TRY(ensure(h->vl_nbr, sizeof(uint16_t) * nn * (size_t)h->vl_cap));
    TRY(ensure(h->vl_ctl, sizeof(int) * 8));
    return MSM_OK;
}

// Size the lists for the system and invalidate them when the system changed or
// the call does not continue a trajectory (fresh): md_run's results then depend
// only on its inputs, never on what the handle ran before.
template <typename T>
static int list_setup(msm_handle *h, const SysDev &s, bool fresh, cudaStream_t st)
{
    TRY(set_geometry(h, s.box, st));
    choose_bricks(h, s.n);
    const double rl = h->p.a + h->p.list_skin, hh = h->p.h;
    const int R = (int)ceil((rl + 1e-3 * hh) / hh) + 1;
    const int rows = (2 * h->bd[1] + 2 * R + 1) * (2 * h->bd[2] + 2 * R + 1);
    const int ngroups = h->nb[0] * ((h->nb[1] + 1) / 2) * ((h->nb[2] + 1) / 2);
    const bool changed = s.n != h->vl_key_n || s.n_mol != h->vl_key_nmol || s.lj != h->vl_key_lj ||
                         memcmp(s.box, h->vl_key_box, sizeof h->vl_key_box) != 0 || rows > h->vl_rows ||
                         ngroups != h->vl_ngroups;
    if (!changed && !fresh && h->vl_ctl.p) return MSM_OK;
    if (h->vl_cap == 0) {
        // entries per atom: pairs within a + skin at 1.8x the box's mean density, at least 256
        double vol = s.box[3] * s.box[4] * s.box[5];
        const double dens = (double)s.n / vol;
        const double want = 1.8 * dens * 4.18879020478639 * rl * rl * rl + 32.0;
        h->vl_cap = ((std::max(256, (int)want) + 7) / 8) * 8;
        h->vl_jcap = sizeof(T) == 4 ? 4608 : 4608;
    }
    h->vl_rows = std::max(h->vl_rows, rows);
    h->vl_ngroups = ngroups;
    TRY(list_alloc(h, s.n, sizeof(vec4<T>)));
    CUDA_TRY(cudaMemsetAsync(h->vl_ctl.p, 0, sizeof(int) * 8, st));
    const int invalid = 1;
    CUDA_TRY(cudaMemcpyAsync(h->vl_ctl.as<int>() + 2, &invalid, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));                    // 'invalid' lives on the host stack
    h->vl_key_n = s.n; h->vl_key_nmol = s.n_mol; h->vl_key_lj = s.lj;
    memcpy(h->vl_key_box, s.box, sizeof h->vl_key_box);
    return MSM_OK;
}

// After an overflow: grow the exceeded capacity, invalidate, resume with lists next time.
static int list_grow(msm_handle *h, cudaStream_t st)
{
    const int *c = h->h_ctl;
    const size_t vsz = h->precision == MSM_FP32 ? sizeof(vec4<float>) : sizeof(vec4<double>);
    const int max_jcap = h->precision == MSM_FP32 ? 10240 : 5120;   // shared memory of one CTA
    if (c[4] + 16 > h->vl_cap) h->vl_cap = (((int)(1.25 * c[4]) + 32 + 7) / 8) * 8;
    if (c[5] > h->vl_jcap) h->vl_jcap = std::min(max_jcap, (((int)(1.2 * c[5]) + 64) + 7) / 8 * 8);
    if (c[6] > h->vl_rows) h->vl_rows = c[6] + 16;
    if (c[5] > max_jcap) h->p.list_skin = 0.0;              // too dense for staged lists: cell search only
    TRY(list_alloc(h, h->vl_key_n, vsz));
    CUDA_TRY(cudaMemsetAsync(h->vl_ctl.p, 0, sizeof(int) * 8, st));
    const int invalid = 1;
    CUDA_TRY(cudaMemcpyAsync(h->vl_ctl.as<int>() + 2, &invalid, sizeof(int), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return MSM_OK;
}

template <typename T> static double shake_tol() { return sizeof(T) == 4 ? 2e-6 : 1e-12; }
template <typename T> static double rattle_tol() { return sizeof(T) == 4 ? 2e-6 : 1e-14; }

// n_steps of velocity Verlet on device arrays; uk (device, nullable) gets
// (U, K) before the first and after every step.  No host synchronisation.
template <typename T>
static int run_md_t(msm_handle *h, const SysDev &s, double dt, int n_steps, double *uk, cudaStream_t st)
{
    const size_t nn = (size_t)(s.n > 0 ? s.n : 1);
    TRY(ensure(h->md_f, sizeof(double) * 3 * nn));
    TRY(ensure(h->md_xo, sizeof(double) * 3 * nn));
    EvalIO io;
    io.n = s.n; io.n_mol = s.n_mol; io.pos = s.x; io.q = s.q; io.lj = s.lj;
    io.forces = s.f ? s.f : h->md_f.as<double>();
    io.pot = nullptr;
    VVArgs va;
    va.n = (int)s.n; va.n_mol = (int)s.n_mol; va.x = s.x; va.v = s.v; va.xo = h->md_xo.as<double>();
    TRY(ensure(h->md_im, sizeof(double) * nn));
    TRY(launch_inverse(int(s.n), s.m, h->md_im.as<double>(), st));
    va.f = io.forces; va.m = s.m; va.im = h->md_im.as<double>(); va.dt = dt;
    va.d_oh2 = h->p.d_oh * h->p.d_oh; va.d_hh2 = h->p.d_hh * h->p.d_hh;
    va.tol = shake_tol<T>(); va.tol_v = rattle_tol<T>(); va.max_iter = sizeof(T) == 4 ? 200 : 1000;
    h->list_on = false;
    if (h->p.list_skin > 0 && s.n > 0) TRY(list_setup<T>(h, s, !(s.f && s.f_valid), st));
    if (s.f && s.f_valid) {
        // forces and energy of the start positions come with the system
        TRY(set_geometry(h, s.box, st));
        TRY(ensure_atoms(h, s.n));
        choose_bricks(h, s.n);
        h->last_n = s.n;
        CUDA_TRY(cudaMemsetAsync(h->status.p, 0, sizeof(int) * 4, st));
        h->h_scal[4] = s.energy;
        CUDA_TRY(cudaMemcpyAsync(h->sums.p, &h->h_scal[4], sizeof(double), cudaMemcpyHostToDevice, st));
    } else {
        TRY(evaluate(h, io, s.box, st));
    }
    va.status = h->status.as<int>();
    if (uk) {
        CUDA_TRY(cudaMemcpyAsync(uk, h->sums.p, sizeof(double), cudaMemcpyDeviceToDevice, st));
        TRY(launch_kinetic(va, h->kin.as<double>(), st));
        const double *cols[1] = {h->kin.as<double>()};
        TRY(launch_sum((int)s.n, 1, cols, h->partials.as<double>(), uk + 1, va.status, st));
    }
    h->list_on = h->vl_ctl.p != nullptr && h->p.list_skin > 0 && s.n > 0;
    for (int step = 0; step < n_steps; step++) {
        { PROF(ST_VV1); TRY(launch_vv_first<T>(va, st)); }
        int rc = evaluate_t<T>(h, io, st);
        if (rc) { h->list_on = false; return rc; }
        { PROF(ST_VV2); TRY(launch_vv_second<T>(va, uk ? h->kin.as<double>() : nullptr, st)); }
        if (uk) {
            CUDA_TRY(cudaMemcpyAsync(uk + 2 * (step + 1), h->sums.p, sizeof(double), cudaMemcpyDeviceToDevice, st));
            const double *cols[1] = {h->kin.as<double>()};
            TRY(launch_sum((int)s.n, 1, cols, h->partials.as<double>(), uk + 2 * (step + 1) + 1, va.status, st));
        }
    }
    h->list_on = false;
    return MSM_OK;
}

static int run_md(msm_handle *h, const SysDev &s, double dt, int n_steps, double *uk, cudaStream_t st)
{
    if (!(dt > 0) || n_steps < 0) return fail_msg(MSM_EINVAL, "dt must be > 0 and n_steps >= 0");
    if (s.n_mol > 0 && h->p.model != MSM_MODEL_WATER) return fail_msg(MSM_EINVAL, "rigid molecules need the water model");
    if (h->precision == MSM_FP32) return run_md_t<float>(h, s, dt, n_steps, uk, st);
    return run_md_t<double>(h, s, dt, n_steps, uk, st);
}

extern "C" int md_run(msm_handle *h, msm_system *sys, double dt, int32_t n_steps, double *uk, void *stream)
{
    if (!h || !sys) return fail_msg(MSM_EINVAL, "handle or system is NULL");
    if (sys->n < 0 || sys->n_mol < 0 || 3 * sys->n_mol > sys->n) return fail_msg(MSM_EINVAL, "bad atom counts");
    if (sys->n > 0 && (!sys->x || !sys->v || !sys->q || !sys->m)) return fail_msg(MSM_EINVAL, "x, v, q, m are required");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nn = (size_t)sys->n;
    SysDev s;
    s.n = sys->n; s.n_mol = sys->n_mol;
    memcpy(s.box, sys->box, sizeof s.box);
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
    if (sys->f) {
        if (f_host) {
            TRY(ensure(h->out_f, sizeof(double) * 3 * nn));
            if (sys->f_valid)
                CUDA_TRY(cudaMemcpyAsync(h->out_f.p, sys->f, sizeof(double) * 3 * nn, cudaMemcpyHostToDevice, st));
            s.f = h->out_f.as<double>();
        } else s.f = sys->f;
        s.f_valid = sys->f_valid;
        s.energy = sys->energy;
    }
    TRY(run_md(h, s, dt, n_steps, ukd, st));
    if (x_host) CUDA_TRY(cudaMemcpyAsync(sys->x, s.x, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (v_host) CUDA_TRY(cudaMemcpyAsync(sys->v, s.v, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (uk_host) CUDA_TRY(cudaMemcpyAsync(uk, ukd, sizeof(double) * ukn, cudaMemcpyDeviceToHost, st));
    if (f_host) CUDA_TRY(cudaMemcpyAsync(sys->f, s.f, sizeof(double) * 3 * nn, cudaMemcpyDeviceToHost, st));
    if (sys->f) CUDA_TRY(cudaMemcpyAsync(&h->h_scal[5], h->sums.p, sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(finish(h, st));
    if (sys->f) { sys->f_valid = 1; sys->energy = h->h_scal[5]; }
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
    ShortArgs<T> s;
    s.g = h->cg;
    for (int d = 0; d < 3; d++) { s.bd[d] = h->bd[d]; s.nb[d] = h->nb[d]; }
    s.nbricks = h->nbricks;
    s.start = h->start.as<int>(); s.apos = h->apos.as<vec4<T>>(); s.aflag = h->aflag.as<int>();
    const double a = h->p.a;
    s.a = (T)a; s.a2 = (T)(a * a); s.a_sel = (T)(a + 1e-3 * h->p.h);
    s.perm = h->perm.as<int>(); s.vl_ctl = nullptr;
    s.sr = nullptr; s.lj = nullptr; s.cnt = h->eatom.as<double>(); s.status = h->status.as<int>();
    CUDA_TRY(cudaMemsetAsync(h->eatom.p, 0, sizeof(double) * (size_t)(h->last_n > 0 ? h->last_n : 1), st));
    TRY(launch_count_pairs<T>(s, st));
    const double *cols[1] = {h->eatom.as<double>()};
    TRY(launch_sum((int)h->last_n, 1, cols, h->partials.as<double>(), h->sums.as<double>() + 2, h->status.as<int>(), st));
    CUDA_TRY(cudaMemcpyAsync(&h->h_scal[3], h->sums.as<double>() + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    TRY(finish(h, st));
    *out = (int64_t)h->h_scal[3];
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

extern "C" int parareal_run(const msm_params *G, double dtG, int32_t stepsG, const msm_params *F, double dtF,
                            int32_t stepsF, const msm_system *state0, int32_t n_slices, int32_t max_iter, double tol,
                            double *slices_x, double *slices_v, int32_t *iters_done, double *last_dx, void *stream)
{
    if (!G || !F || !state0 || !slices_x || !slices_v) return fail_msg(MSM_EINVAL, "NULL argument");
    if (n_slices < 1 || max_iter < 0 || stepsG < 0 || stepsF < 0 || !(tol >= 0))
        return fail_msg(MSM_EINVAL, "bad parareal sizes");
    if (fabs(dtG * stepsG - dtF * stepsF) > 1e-9 * fabs(dtF * stepsF))
        return fail_msg(MSM_EINVAL, "G and F must span the same slice length");
    const msm_system &s0 = *state0;
    if (s0.n <= 0 || !s0.x || !s0.v || !s0.q || !s0.m) return fail_msg(MSM_EINVAL, "state0 incomplete");
    cudaStream_t st = (cudaStream_t)stream;
    msm_handle *hG = nullptr, *hF = nullptr;
    TRY(msm_create(G, &hG));
    int rc = msm_create(F, &hF);
    if (rc) { msm_destroy(hG); return rc; }
    const size_t n3 = 3 * (size_t)s0.n, nn = (size_t)s0.n, ns = (size_t)n_slices;
    DevBuf lam_x, lam_v, new_x, new_v, gold_x, gold_v, f_x, f_v, tmp_x, tmp_v, q, m, lj, part, dx;
    auto cleanup = [&]() {
        DevBuf *all[] = {&lam_x, &lam_v, &new_x, &new_v, &gold_x, &gold_v, &f_x, &f_v, &tmp_x, &tmp_v, &q, &m, &lj, &part, &dx};
        for (DevBuf *b : all) release(*b);
        msm_destroy(hG);
        msm_destroy(hF);
    };
    auto body = [&]() -> int {
        TRY(ensure(lam_x, sizeof(double) * n3 * (ns + 1)));
        TRY(ensure(lam_v, sizeof(double) * n3 * (ns + 1)));
        TRY(ensure(new_x, sizeof(double) * n3 * (ns + 1)));
        TRY(ensure(new_v, sizeof(double) * n3 * (ns + 1)));
        TRY(ensure(gold_x, sizeof(double) * n3 * ns));
        TRY(ensure(gold_v, sizeof(double) * n3 * ns));
        TRY(ensure(f_x, sizeof(double) * n3 * ns));
        TRY(ensure(f_v, sizeof(double) * n3 * ns));
        TRY(ensure(tmp_x, sizeof(double) * n3));
        TRY(ensure(tmp_v, sizeof(double) * n3));
        TRY(ensure(q, sizeof(double) * nn));
        TRY(ensure(m, sizeof(double) * nn));
        TRY(ensure(lj, nn));
        const size_t nblk = (n3 + 255) / 256;
        TRY(ensure(part, sizeof(double) * nblk * ns));
        TRY(ensure(dx, sizeof(double)));
        CUDA_TRY(cudaMemcpyAsync(lam_x.p, s0.x, sizeof(double) * n3, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(lam_v.p, s0.v, sizeof(double) * n3, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(q.p, s0.q, sizeof(double) * nn, cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(m.p, s0.m, sizeof(double) * nn, cudaMemcpyDefault, st));
        if (s0.lj) CUDA_TRY(cudaMemcpyAsync(lj.p, s0.lj, nn, cudaMemcpyDefault, st));
        else CUDA_TRY(cudaMemsetAsync(lj.p, 0, nn, st));
        auto X = [&](DevBuf &b, size_t k) { return b.as<double>() + k * n3; };
        SysDev sd;
        sd.n = s0.n; sd.n_mol = s0.n_mol; sd.q = q.as<double>(); sd.m = m.as<double>(); sd.lj = lj.as<uint8_t>();
        memcpy(sd.box, s0.box, sizeof sd.box);
        auto run = [&](msm_handle *hh, double *x, double *v, double dt, int steps) -> int {
            SysDev t = sd;
            t.x = x; t.v = v;
            TRY(run_md(hh, t, dt, steps, nullptr, st));
            return finish(hh, st);
        };
        // init row: lambda^0_{n+1} = G(lambda^0_n)
        for (size_t k = 0; k < ns; k++) {
            CUDA_TRY(cudaMemcpyAsync(tmp_x.p, X(lam_x, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(tmp_v.p, X(lam_v, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            TRY(run(hG, tmp_x.as<double>(), tmp_v.as<double>(), dtG, stepsG));
            CUDA_TRY(cudaMemcpyAsync(X(gold_x, k), tmp_x.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(X(gold_v, k), tmp_v.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(X(lam_x, k + 1), tmp_x.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(X(lam_v, k + 1), tmp_v.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
        }
        int done = 0;
        double dxh = INFINITY;
        for (int it = 0; it < max_iter; it++) {
            // f_n = F(lambda^k_n) for every slice (independent)
            for (size_t k = 0; k < ns; k++) {
                CUDA_TRY(cudaMemcpyAsync(X(f_x, k), X(lam_x, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
                CUDA_TRY(cudaMemcpyAsync(X(f_v, k), X(lam_v, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
                TRY(run(hF, X(f_x, k), X(f_v, k), dtF, stepsF));
            }
            // sequential correction sweep
            CUDA_TRY(cudaMemcpyAsync(new_x.p, lam_x.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            CUDA_TRY(cudaMemcpyAsync(new_v.p, lam_v.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            for (size_t k = 0; k < ns; k++) {
                CUDA_TRY(cudaMemcpyAsync(tmp_x.p, X(new_x, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
                CUDA_TRY(cudaMemcpyAsync(tmp_v.p, X(new_v, k), sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
                TRY(run(hG, tmp_x.as<double>(), tmp_v.as<double>(), dtG, stepsG));
                TRY(launch_parareal_update((int)n3, X(f_x, k), tmp_x.as<double>(), X(gold_x, k), X(new_x, k + 1),
                                           X(lam_x, k + 1), part.as<double>() + k * nblk, st));
                TRY(launch_parareal_update((int)n3, X(f_v, k), tmp_v.as<double>(), X(gold_v, k), X(new_v, k + 1),
                                           nullptr, nullptr, st));
                CUDA_TRY(cudaMemcpyAsync(X(gold_x, k), tmp_x.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
                CUDA_TRY(cudaMemcpyAsync(X(gold_v, k), tmp_v.p, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st));
            }
            TRY(launch_max_reduce((int)(nblk * ns), part.as<double>(), dx.as<double>(), st));
            CUDA_TRY(cudaMemcpyAsync(&hF->h_scal[0], dx.p, sizeof(double), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            dxh = hF->h_scal[0];
            std::swap(lam_x, new_x);
            std::swap(lam_v, new_v);
            done = it + 1;
            if (dxh <= tol) break;
        }
        CUDA_TRY(cudaMemcpyAsync(slices_x, lam_x.p, sizeof(double) * n3 * (ns + 1), cudaMemcpyDefault, st));
        CUDA_TRY(cudaMemcpyAsync(slices_v, lam_v.p, sizeof(double) * n3 * (ns + 1), cudaMemcpyDefault, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (iters_done) *iters_done = done;
        if (last_dx) *last_dx = dxh;
        if (max_iter > 0 && !(dxh <= tol)) return fail_msg(MSM_ENOCONV, "parareal: max |dx| = %g after %d iterations", dxh, done);
        return MSM_OK;
    };
    rc = body();
    cleanup();
    return rc;
}

// -------------------------------------------------------------- inspection

extern "C" int msm_grid_shape(msm_handle *h, int32_t level, int64_t shape[3], int64_t lo[3])
{
    if (!h || !h->have_geom) return fail_msg(MSM_EINVAL, "no evaluation yet");
    if (level < 0 || level >= h->gg.levels) return fail_msg(MSM_EINVAL, "level out of range");
    for (int d = 0; d < 3; d++) {
        if (shape) shape[d] = h->gg.L[level].n[d];
        if (lo) lo[d] = h->gg.L[level].lo[d];
    }
    return MSM_OK;
}

extern "C" int msm_stage_grid(msm_handle *h, int32_t level, int32_t which, double *out, int64_t count)
{
    if (!h || !h->have_geom || !out) return fail_msg(MSM_EINVAL, "no evaluation yet");
    const int l = h->gg.levels;
    if (level < 0 || level >= l || which < 0 || which > 2 || (which == 1 && level == l - 1))
        return fail_msg(MSM_EINVAL, "no such grid");
    const LevelGeom &L = h->gg.L[level];
    const int64_t m = (int64_t)L.n[0] * L.n[1] * L.n[2];
    if (count < m) return fail_msg(MSM_EINVAL, "output too small");
    CUDA_TRY(cudaDeviceSynchronize());
    if (which == 2 && level == l - 1) {
        CUDA_TRY(cudaMemcpy(out, h->utop.p, sizeof(double) * m, cudaMemcpyDeviceToHost));
        return MSM_OK;
    }
    const DevBuf &b = which == 0 ? h->qgrid : (which == 1 ? h->ucut : h->ugrid);
    if (h->precision == MSM_FP64) {
        CUDA_TRY(cudaMemcpy(out, b.as<double>() + L.off, sizeof(double) * m, cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp((size_t)m);
        CUDA_TRY(cudaMemcpy(tmp.data(), b.as<float>() + L.off, sizeof(float) * m, cudaMemcpyDeviceToHost));
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
    const int64_t v[8] = {h->vl_builds, h->vl_overflows, h->vl_cap, h->vl_jcap, h->vl_rows,
                          h->vl_seen[0], h->vl_seen[1], h->vl_seen[2]};
    for (int k = 0; k < 8 && k < max; k++) out[k] = v[k];
    return MSM_OK;
}

extern "C" int64_t msm_kernel_launches(void) { return g_launches.load(); }

extern "C" const char *msm_last_error(void) { return g_err; }
