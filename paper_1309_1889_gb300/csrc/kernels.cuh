// kernels.cuh -- argument blocks and host launchers of every kernel in
// libmsm_gb300.so (internal; the C ABI is include/msm.h).
#pragma once

#include "common.cuh"

namespace msm {

// ---- binning (k_bin.cu) --------------------------------------------------
template <typename T> struct BinArgs {
    int n;
    const double *pos;     // n*3 FP64, original order
    const double *q;       // n
    const uint8_t *lj;     // n, nullable
    CellGeom g;
    double inv_h;          // 1/h rounded once in FP64 (the binning contract)
    int *key;              // n
    int *count;            // ncells + 1 (histogram, left zeroed by the scatter)
    int *start;            // ncells + 1
    int *perm;             // n: sorted slot -> atom
    int *bsum;             // scan scratch (scan_scratch_ints())
    vec4<T> *rel;          // n, original order: (x - x0, y - y0, z - z0, q)
    vec4<T> *frac;         // n, original order: fractional position in the cell, q
    vec4<T> *apos;         // n, sorted copy of rel
    vec4<T> *afrac;        // n, sorted copy of frac
    int *akey;             // n, sorted key
    int *aflag;            // n, sorted (molecule id << 1) | LJ flag
    int n_mol;             // leading rigid triples: atom i < 3 n_mol belongs to molecule i / 3
    int *status;
};
template <typename T> int launch_bin(const BinArgs<T> &a, cudaStream_t st);
int scan_scratch_ints();
int launch_sort_by_key(int n, int m, const int *key, int *count, int *start, int *perm, int *bsum, int *status,
                       cudaStream_t st);

// ---- short range (k_short.cu) ----------------------------------------------
template <typename T> struct ShortArgs {
    CellGeom g;
    int bd[3];             // brick edge in cells
    int nb[3];             // bricks per axis
    int nbricks;
    const int *start;      // cell_start
    const vec4<T> *apos;
    const int *aflag;
    T a, a2, a_sel;        // cutoff, its square, row-selection radius (cutoff + rounding pad)
    T c0, c1, c2;          // gamma(r/a)/a = c0 + c1 r^2 + c2 r^4
    T d0, d1;              // -g*'(r)/r - 1/r^3 = d0 + d1 r^2
    T lj_s2, lj_4eps, lj_24eps, lj_shift;
    const int *perm;       // sorted slot -> atom
    vec4<T> *sr;           // by atom: (F_x, F_y, F_z, phi) of the g* sum, before k_e
    vec4<T> *lj;           // by atom: (F_x, F_y, F_z, E) of the LJ sum (nullable)
    double *cnt;           // counting mode: per sorted atom, number of j with r_ij < a
    const int *vl_ctl;     // Verlet-list flags (nullable): skip when the list path ran
    const int *status;
};
// model = true: skip pairs of the same molecule (their smooth part is removed by
// the exclusion kernel) and add the LJ term between flagged sites.
template <typename T> int launch_short(const ShortArgs<T> &a, bool model, cudaStream_t st);
template <typename T> int launch_count_pairs(const ShortArgs<T> &a, cudaStream_t st);

// ---- Verlet lists (k_list.cu) --------------------------------------------
template <typename T> struct ListArgs {
    CellGeom g;
    int bd[3], nb[3];      // bricks of the short-range kernel
    int ng[3], ngroups;    // groups of 1 x 2 x 2 bricks
    int max_rows, jcap, cap;   // row slots per group, staged atoms per group, list entries per atom
    T a2, rl2, rl_sel, skin_half2;
    T c0, c1, c2, d0, d1;
    T lj_s2, lj_4eps, lj_24eps, lj_shift;
    bool model;
    int n;
    const double *x, *q;   // this step, original order
    const int *perm, *start;
    const vec4<T> *apos;
    const int *aflag;
    int *vl_perm, *vl_start;   // reference order of the last build
    double *vl_xref;
    vec4<T> *vl_pos;
    int2 *grp_rows;
    int *grp_nrows, *grp_j;
    int *cnt, *cntlj;
    uint16_t *nbr;         // n x cap
    int *ctl;
    vec4<T> *sr, *lj;      // outputs by atom
    const int *status;
};
template <typename T> int launch_list_maintain(const ListArgs<T> &a, cudaStream_t st);
template <typename T> int launch_list_force(const ListArgs<T> &a, cudaStream_t st);

// ---- grids (k_grid.cu) -----------------------------------------------------
template <typename T> struct AnterpArgs {
    CellGeom cg;
    LevelGeom L0;
    const int *start;
    const vec4<T> *afrac;
    T *q0;
    const int *status;
};
template <typename T> int launch_anterp(const AnterpArgs<T> &a, cudaStream_t st);

template <typename T> int launch_restrict(const LevelGeom &fine, const LevelGeom &coarse, const T *qf, T *qc,
                                          const int *status, cudaStream_t st);

struct StencilGeom {
    int rad;               // max |n_x| of a tap: largest r with r h < 2a
    int wdim;              // 2 rad + 1
    int nrows;             // non-empty (dy, dz) rows
};
template <typename T> struct StencilArgs {
    GridGeom gg;
    int nlev;              // levels 0..nlev-1 get a lattice cutoff (nlev = l - 1)
    int blk_off[MSM_MAX_LEVELS + 1];
    int tiles[MSM_MAX_LEVELS][3];
    StencilGeom sg;
    const T *w;            // wdim^3 weights g^0(|n| h) (0 outside the sphere), x fastest
    const int4 *rows;      // (dy, dz, half-width, 0) of each non-empty row
    const T *q;            // concatenated grids (GridGeom offsets)
    T *ucut;               // concatenated, levels < nlev
    const int *status;
};
template <typename T> int launch_stencil(const StencilArgs<T> &a, int *tile_counter, cudaStream_t st);
template <typename T> size_t stencil_smem_bytes(int rad);

int launch_top_table(const LevelGeom &top, double a_top, double h_top, double *table, cudaStream_t st);
template <typename T> int launch_top(const LevelGeom &top, const double *table, const T *qtop, double *utop,
                                     const int *status, cudaStream_t st);
// uc points at the first point of the coarse level (its own array or an offset
// into the concatenated grids); ucut and uf are concatenated (fine.off applies).
template <typename T, typename S> int launch_prolong(const LevelGeom &fine, const LevelGeom &coarse, const T *ucut,
                                                      const S *uc, T *uf, const int *status, cudaStream_t st);
void stencil_tiles(const LevelGeom &L, int t[3]);
int launch_cast_f64(int m, const double *src, float *dst, cudaStream_t st);
int launch_stencil_table(double a, double h, int rad, double *wd, cudaStream_t st);

template <typename T> struct InterpArgs {
    int n;
    CellGeom cg;
    LevelGeom L0;
    const int *perm;
    const int *akey;
    const vec4<T> *afrac;
    const vec4<T> *sr;
    const vec4<T> *lj;     // nullable
    const T *u0;
    const double *pos;     // n*3, original order (virial)
    const double *q;       // n, original order
    double ke, self;       // k_e, gamma(0)/a
    double inv_h;
    double box_lo[3], box_hi[3];   // domain faces (wall of the water completion)
    double wall_k, wall_w;         // wall_k = 0: no wall
    double *forces;        // n*3, original order (nullable)
    double *pot;           // n (nullable)
    double *eatom;         // n: 1/2 q_i phi_i + 1/2 E_lj,i
    double *vatom;         // n: r_i . F_i
    const int *status;
};
template <typename T> int launch_interp(const InterpArgs<T> &a, cudaStream_t st);

// ---- dynamics and reductions (k_md.cu) -------------------------------------
struct ExclArgs {
    int n_mol;
    const double *x;
    const double *q;
    double ke, a;
    double *forces, *pot, *eatom, *vatom;
    const int *status;
};
template <typename T> int launch_exclusions(const ExclArgs &a, cudaStream_t st);

// Deterministic FP64 sum of m values per column (ncols arrays) into out[ncols].
int launch_sum(int m, int ncols, const double *const *cols, double *partials, double *out, const int *status,
               cudaStream_t st);
int sum_partials_needed(int m);

struct VVArgs {
    int n, n_mol;
    double *x, *v;
    double *xo;            // scratch: positions before the drift
    const double *f, *m;
    const double *im;      // 1/m, computed once per md_run call
    double dt;
    double d_oh2, d_hh2;
    double tol;            // relative tolerance on squared bond lengths (SHAKE)
    double tol_v;          // absolute tolerance on (v_i - v_j).(x_i - x_j) (RATTLE), nm^2/ps
    int max_iter;
    int *status;
};
template <typename T> int launch_vv_first(const VVArgs &a, cudaStream_t st);
template <typename T> int launch_vv_second(const VVArgs &a, double *kin_atom, cudaStream_t st);
int launch_kinetic(const VVArgs &a, double *kin_atom, cudaStream_t st);
int launch_inverse(int n, const double *m, double *im, cudaStream_t st);

int launch_parareal_update(int count, const double *f, const double *gnew, const double *gold, double *out,
                           const double *prev, double *dx_partials, cudaStream_t st);
int launch_max_reduce(int m, const double *v, double *out, cudaStream_t st);

}  // namespace msm
