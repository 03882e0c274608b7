// kernels.cuh -- argument blocks and host launchers of every kernel in
// libmsm_gb300.so (internal; the C ABI is include/msm.h).
#pragma once

#include <cuda.h>          // CUtensorMap: TMA descriptors of the lattice-cutoff planes

#include "common.cuh"

namespace msm {

// ---- batch launch shape ----------------------------------------------------
// Every batched kernel runs on a grid (x, B): blockIdx.y is the system and
// blocks past that system's work return at once.  gx is the x extent needed
// by the largest system.
struct Batch {
    int B;                 // systems
    const SysDesc *sd;     // device array of B descriptors
};

// ---- binning (k_bin.cu) --------------------------------------------------
template <typename T> struct BinArgs {
    Batch bt;
    int n_total;           // atoms over all systems
    int m_total;           // cells over all systems
    int max_n;             // atoms of the largest system
    const double *pos;     // n_total*3 FP64, original order (systems concatenated)
    const double *q;       // n_total
    const uint8_t *lj;     // n_total, nullable
    int *key;              // n_total: global cell id (system cell_off + local key)
    int *count;            // m_total + 1 (histogram, left zeroed by the scatter)
    int *start;            // m_total + 1
    int *perm;             // n_total: sorted slot -> atom
    int *bsum;             // scan scratch (scan_scratch_ints(m_total))
    vec4<T> *rel;          // original order: (x - x0, y - y0, z - z0, q) of the atom's system
    vec4<T> *frac;         // original order: fractional position in the cell, q
    vec4<T> *apos;         // sorted copy of rel
    vec4<T> *afrac;        // sorted copy of frac
    int *akey;             // sorted global cell id
    int *aflag;            // sorted (molecule id << 1) | LJ flag; molecule id = global
                           // index of the molecule's first atom (single sites: own index)
    vec4<T> *aw;           // sorted anterpolation weights, 3 n_total: [0, n) q wx[0..3],
                           // [n, 2n) wy[0..3], [2n, 3n) wz[0..3]
    int *status;
};
template <typename T> int launch_bin(const BinArgs<T> &a, cudaStream_t st);
int scan_scratch_ints(int m);             // scratch ints of a scan of m values
int launch_diag_convert(int64_t n, const double *x, float *x32, const float *y, double *y64, cudaStream_t st);
int launch_scan(int m, const int *count, int *start, int *bsum, const int *status, cudaStream_t st);
int launch_sort_by_key(int n, int m, const int *key, int *count, int *start, int *perm, int *bsum, int *status,
                       cudaStream_t st);

// ---- short range (k_short.cu) ----------------------------------------------
template <typename T> struct ShortArgs {
    Batch bt;
    int max_bricks;        // bricks of the largest system (of its LJ pass for launch_short_lj)
    const int *start;      // global cell_start
    const vec4<T> *apos;
    const int *aflag;
    T a, a2, a_sel;        // cutoff, its square, row-selection radius (cutoff + rounding pad)
    T c0, c1, c2;          // gamma(r/a)/a = c0 + c1 r^2 + c2 r^4
    T d0, d1;              // -g*'(r)/r - 1/r^3 = d0 + d1 r^2
                           // (all five 0 for the simple cutoff: the pair term is 1/r)
    bool wolf;             // Wolf summation: pair term erfc(alpha r)/r - w_shift
    T w_alpha, w_shift, w_c;   // alpha, erfc(alpha a)/a, 2 alpha/sqrt(pi)
    T lj_s2, lj_4eps, lj_24eps, lj_shift;
    const int *perm;       // sorted slot -> atom
    vec4<T> *sr;           // by atom: (F_x, F_y, F_z, phi) of the g* sum, before k_e
    vec4<T> *lj;           // by atom: (F_x, F_y, F_z, E) of the LJ sum (nullable)
    double *cnt;           // counting mode: per sorted atom, number of j with r_ij < a
    const int *vl_ctl;     // Verlet-list flags (nullable): skip when the list path ran
    const int *status;
    bool scalar_pairs;     // FP32 pair passes: one queued j per step instead of packed pairs
    // i groups (nullable: bricks): per global column the first group (scan of the group
    // counts, columns + 1 entries), and 32 sorted slots per group (-1: no atom)
    const int *gcol;
    const int *gslot;
};
// i groups of the pair passes: each column of cw x cw cells (SysDesc::gp_* or, lj,
// lgp_*) has ceil(atoms / 32) groups, its atoms taken layer by layer (each layer
// in ascending z) and cut into runs of 32.  gcnt, gcol: columns + 1 entries;
// bsum: scan scratch; apos: the sorted positions the cell starts index; max_cols,
// max_nz: columns and cell layers of the largest system.
template <typename T>
int launch_groups(const Batch &bt, bool lj, int max_cols, int max_nz, int n_cols, const int *start,
                  const vec4<T> *apos, int *gcnt, int *gcol, int *bsum, int *gslot, const int *status, cudaStream_t st);
// model = true: skip pairs of the same molecule (their smooth part is removed by
// the exclusion kernel) and write a zero LJ output for atoms that are not LJ
// sites; the LJ term itself is the separate pass below.
template <typename T> int launch_short(const ShortArgs<T> &a, bool model, cudaStream_t st);
// O-O Lennard-Jones of the water completion over the LJ sites only: a the
// ShortArgs of the LJ-site cell list (start, apos, aflag, perm of the subset),
// bricks from SysDesc::lj_*; writes lj[atom] of every LJ site.
template <typename T> int launch_short_lj(const ShortArgs<T> &a, cudaStream_t st);
// The LJ-site cell list: per global cell the LJ sites among its sorted slots,
// compacted in slot order (count -> lj_start by launch_scan -> copies).
template <typename T> int launch_lj_count(int m_total, const int *start, const int *aflag, int *lj_count,
                                          const int *status, cudaStream_t st);
template <typename T> int launch_lj_compact(int m_total, const int *start, const int *lj_start, const vec4<T> *apos,
                                            const int *aflag, const int *perm, vec4<T> *lj_apos, int *lj_flag,
                                            int *lj_perm, const int *status, cudaStream_t st);
template <typename T> int launch_count_pairs(const ShortArgs<T> &a, cudaStream_t st);

// ---- cluster pairs (k_cluster.cu, FP32) -------------------------------------
// Columns of 2 x 2 finest cells per system (SysDesc::cp_nc, col_off, zc_off);
// clusters of 4 atoms in column order, two per i cluster of 8.
struct ClusterArgs {
    Batch bt;
    int max_cols;          // columns of the largest system
    int n_cols;            // columns over all systems
    int max_icl;           // bound on the i clusters of the largest system (n/8 + columns)
    const int *start;      // global cell_start
    const vec4<float> *apos;
    const int *aflag;
    const int *perm;
    int *col_n;            // n_cols: clusters of 4 per column (even)
    int *col_cl;           // n_cols + 1: first cluster of 4 of each column (scan of col_n)
    int *bsum;             // scan scratch (scan_scratch_ints(n_cols))
    int *zc;               // per column, nz + 1 entries: atoms of the column below cell layer z
    vec4<float> *cpos;     // 4 per cluster: (x, y, z, q), padding (-1000, -1000, -1000, 0)
    int *cmol;             // 4 per cluster: molecule id (water model), padding -2
    int *cslot;            // 4 per cluster: sorted slot, padding -1
    vec4<float> *cbox;     // 2 per cluster: low and high corner of its atoms
    float a, a2, a_sel;
    float c0, c1, c2, d0, d1;   // as ShortArgs
    vec4<float> *sr;       // by atom: (F_x, F_y, F_z, phi) of the g* sum, before k_e
    vec4<float> *lj;       // water model: zeroed for atoms that are not LJ sites
    const int *vl_ctl;
    const int *status;
};
// k_cp_count, the scan of the column counts, k_cp_fill
int launch_cluster_build(const ClusterArgs &a, bool model, cudaStream_t st);
// the Coulomb pass on cluster pairs (model: rigid-water exclusions, as launch_short)
int launch_cluster_short(const ClusterArgs &a, bool model, cudaStream_t st);

// ---- Verlet lists (k_list.cu, single systems) -----------------------------
constexpr int VL_ROWS = 512;       // candidate rows per brick (9 bits of an entry)
constexpr int VL_OFFS = 128;       // atoms per row segment (7 bits of an entry)
template <typename T> struct ListArgs {
    CellGeom g;
    int bd[3], nb[3], nbricks; // bricks of the short-range kernel (frozen with the list)
    int cap, cap_lj;       // entries per atom (multiples of 4): all partners, O-O partners
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
    vec4<T> *vl_pos;       // this step's positions in reference order
    int *rtab;             // nbricks x VL_ROWS: first reference slot of each candidate row
    int *rtn;              // nbricks: candidate rows of each brick
    int *cnt, *cntlj;      // entries per reference slot
    unsigned long long *nbr, *nbr_lj;   // entry quads: quad q of slot s at [q * n + s]
    int *ctl;
    vec4<T> *sr, *lj;      // outputs by atom
    const int *status;
};
template <typename T> int launch_list_maintain(const ListArgs<T> &a, cudaStream_t st);
template <typename T> int launch_list_force(const ListArgs<T> &a, cudaStream_t st);

// ---- grids (k_grid.cu) -----------------------------------------------------
template <typename T> struct AnterpArgs {
    Batch bt;
    int max_tiles;         // anterpolation tiles of the largest level-0 grid
    int n_total;           // atoms over all systems (stride of the weight records)
    const int *start;      // global cell_start
    const vec4<T> *aw;     // sorted weight records (BinArgs::aw)
    T *q;                  // concatenated grids
    const int *status;
};
template <typename T> int launch_anterp(const AnterpArgs<T> &a, cudaStream_t st);
int anterp_tiles(const LevelGeom &L0);

// level k -> k+1 of every system; max_coarse = points of the largest level k+1
template <typename T> int launch_restrict(const Batch &bt, int k, int max_coarse, T *q, const int *status,
                                          cudaStream_t st);

struct StencilGeom {
    int rad;               // max |n_x| of a tap: largest r with r h < 2a
    int wdim;              // 2 rad + 1
    int nrows;             // non-empty (dy, dz) rows
    int plane;             // values of one shared-memory plane buffer (largest tile of the batch)
};
template <typename T> struct StencilArgs {
    Batch bt;
    int nlev;              // levels 0..nlev-1 get a lattice cutoff (nlev = l - 1)
    const int *blk_off;    // B*nlev + 1 tile offsets, entry s*nlev + k = first tile of (system s, level k)
    int total_tiles;
    StencilGeom sg;
    const T *w;            // wdim^3 weights g^0(|n| h) (0 outside the sphere), x fastest
    const int4 *rows;      // (dy, dz, half-width, 0) of each non-empty row
    const T *q;            // concatenated grids
    T *ucut;               // concatenated, levels < nlev
    size_t ucut_len;       // values of ucut zeroed before the two plane halves of each tile add into it
    const int *status;
};
// maps: one TMA descriptor per (system, level) entry of the batch (encode_stencil_maps);
// blk: the host copy of blk_off.  Entries are launched in groups of at most
// ST_MAXMAPS, each group's descriptors passed as a kernel parameter.
template <typename T> int launch_stencil(const StencilArgs<T> &a, const CUtensorMap *maps, const int *blk,
                                         int *tile_counter, cudaStream_t st);
// Encode the descriptors of every (system s, level k < nlev) of a batch into
// maps[s*nlev + k]: 3-D tiled maps of level k's grid inside q (rows of n[0], a
// multiple of 4 values), box = one plane of a tile with its halos, zero fill.
template <typename T> int encode_stencil_maps(const SysDesc *sd, int B, int nlev, int rad, const T *q,
                                              CUtensorMap *maps);
template <typename T> size_t stencil_smem_bytes(int rad, int plane);
int stencil_tile_count(const LevelGeom &L);
int stencil_plane_values(const LevelGeom &L, int rad);   // plane buffer a tile of level L needs

int launch_top_table(const LevelGeom &top, double a_top, double h_top, double *table, cudaStream_t st);
// utop: per system top_off; max_top = points of the largest top level
template <typename T> int launch_top(const Batch &bt, int max_top, const double *table, const T *q, double *utop,
                                     const int *status, cudaStream_t st);
// u^k = u^{k,cut} + prolongation of u^{k+1} for level k of every system; the
// coarse level is the FP64 top buffer when from_top, else the grid buffer.
template <typename T> int launch_prolong(const Batch &bt, int k, int max_fine, const T *ucut, const double *utop,
                                         bool from_top, T *u, const int *status, cudaStream_t st);
// l = 1: the top level is level 0; copy it (to the compute type) into u.
template <typename T> int launch_top_to_grid(const Batch &bt, int max_top, const double *utop, T *u,
                                             const int *status, cudaStream_t st);
int launch_cast_f64(int m, const double *src, float *dst, cudaStream_t st);
int launch_stencil_table(double a, double h, int rad, double *wd, cudaStream_t st);

template <typename T> struct InterpArgs {
    Batch bt;
    int max_n;
    const int *perm;
    const int *akey;       // global cell ids
    const vec4<T> *afrac;
    const vec4<T> *sr;
    const vec4<T> *lj;     // nullable
    const T *u;            // concatenated grids (NULL: no grid part, the cutoff methods)
    const double *pos;     // original order (virial, wall)
    const double *q;       // original order
    double ke, self;       // k_e, self coefficient: phi_i -= q_i self (gamma(0)/a for the MSM)
    double wall_k, wall_w; // wall_k = 0: no wall
    double *forces;        // original order (nullable)
    double *pot;           // (nullable)
    double *eatom;         // 1/2 q_i phi_i + 1/2 E_lj,i
    double *vatom;         // r_i . F_i
    // multiple time stepping, split evaluation (both NULL otherwise): forces then
    // receives the fast part (pair sum, LJ, wall), fslow the grid part
    // -k_e q_i grad u^long, eslow the slow energy 1/2 q_i k_e (u_i^long - q_i self)
    double *fslow, *eslow;
    const int *status;
};
template <typename T> int launch_interp(const InterpArgs<T> &a, cudaStream_t st);

// ---- dynamics and reductions (k_md.cu) -------------------------------------
struct ExclArgs {
    Batch bt;
    int max_mol;
    const double *x;
    const double *q;
    double ke, a, inv_a;   // k_e, a and 1/a (rounded once, FP64)
    double *forces, *pot, *eatom, *vatom;
    double *fslow, *eslow; // split evaluation: the correction's forces go to fslow (not forces),
                           // its energy to eslow as well (both NULL otherwise)
    const int *status;
};
template <typename T> int launch_exclusions(const ExclArgs &a, cudaStream_t st);

// Deterministic FP64 sums, per system: column c of system s sums its n values
// in fixed chunks of SUM_CHUNK atoms (the same partition whatever the batch)
// and writes out[s * out_stride + c].  part holds ncols * total_blocks values.
int launch_sum(const Batch &bt, int max_n, int total_blocks, int ncols, const double *const *cols, double *part,
               double *out, int out_stride, const int *status, cudaStream_t st);
__host__ __device__ int sum_blocks(int n);

struct VVArgs {
    Batch bt;
    int max_units;         // molecules + single sites of the largest system
    double *x, *v;
    double *xo;            // scratch: positions before the drift
    const double *f, *m;
    const double *fs;      // multiple time stepping: the kicks use f + ws * fs (NULL: f alone)
    double ws;
    const double *im;      // 1/m, computed once per md_run call
    double dt;
    double d_oh2, d_hh2;
    double tol;            // relative tolerance on squared bond lengths (SHAKE)
    double tol_v;          // RATTLE tolerance on (v_i - v_j).(x_i - x_j): absolute (nm^2/ps) in FP64,
                           // relative to |x_i - x_j| (|v_i| + |v_j|) in FP32
    int max_iter;
    int *status;           // on a constraint failure status[1] = 1 (SHAKE) or 2 (RATTLE) and
                           // status[3] = 1 + the molecule's first atom
};
template <typename T> int launch_vv_first(const VVArgs &a, cudaStream_t st);
template <typename T> int launch_vv_second(const VVArgs &a, double *kin_atom, cudaStream_t st);
int launch_kinetic(int n, const double *v, const double *m, double *kin_atom, cudaStream_t st);
int launch_inverse(int n, const double *m, double *im, cudaStream_t st);
// uk[s][step][2] <- (U_s, K_s) for every system; step from *ctr, then ++*ctr.  With add_slow
// U_s = sums[s][0] + sums[s][2] (a fast-only evaluation plus the last slow energy).
int launch_record_uk(int B, const double *sums, int sums_stride, const double *kin, double *uk, int uk_stride,
                     int *ctr, bool add_slow, cudaStream_t st);
// y[i] += x[i], i < n (FP64)
int launch_add(int64_t n, const double *x, double *y, cudaStream_t st);

int launch_parareal_update(int count, const double *f, const double *gnew, const double *gold, double *out,
                           const double *prev, double *dx_partials, cudaStream_t st);
int launch_max_reduce(int m, const double *v, double *out, cudaStream_t st);
// Rigid-molecule projection of a corrected parareal state (x, v of n_mol leading triples).
int launch_pr_project(int n_mol, double *x, double *v, const double *m, double d_oh2, double d_hh2, double thresh,
                      double tol, double tol_v, int *status, cudaStream_t st);
int launch_absdiff_partials(int count, const double *a, const double *b, double *part, cudaStream_t st);
// out[s] = max of v[s*m .. s*m + m), s < nseg.
int launch_max_reduce_seg(int nseg, int m, const double *v, double *out, cudaStream_t st);
// First failure of a sequence of propagations: dst = (code, kind, tag, atom + 1) of src once.
int launch_status_fold(const int *src, int *dst, int tag, cudaStream_t st);

}  // namespace msm
