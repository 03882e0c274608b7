// k_short.cu -- short-range part of the MSM (Sec. 3, step 1):
//   u_i^short = sum_{j != i, r_ij < a} q_j g*(r_ij),  g*(r) = 1/r - gamma(r/a)/a,
//   F_i^short = -q_i sum_j q_j g*'(r_ij) (r_i - r_j)/r_ij
//             =  q_i sum_j q_j [1/r^3 - 5/(2a^3) + 3r^2/(2a^5)] (r_i - r_j).
// The same kernel sums the pair terms of the coarse propagators of Sec. 5:
// the simple cutoff (g = 1/r: the gamma coefficients are zero) and Wolf
// summation (g = erfc(alpha r)/r - erfc(alpha a)/a, the WOLF instance).
//
// Layout: atoms sorted by finest-grid cell (x fastest), so a run of cells
// along x is one contiguous slot range.  One warp owns one group of 32 i atoms
// (one per lane): the cells are grouped into columns of cw x cw cells (cw^3
// cells hold ~32 atoms at the mean density), and each column's atoms, layer by
// layer and in ascending z inside a layer, are cut into runs of 32
// (k_grp_count, k_grp_fill).  Every
// lane has an atom, and the groups' bounding boxes are compact: ~2.7 candidate
// evaluations per pair within a on water, against ~3.3 for bricks.  With
// MSM_FLAG_BRICKS the warp owns a brick of bd[0] x bd[1] x bd[2] cells instead
// (about 20 atoms, taken 32 at a time).  The warp's j candidates are whole cell rows (fixed y, z) whose distance to the
// bounding box of its i atoms is below a, each trimmed in x to the cells that
// can still lie within a: every row is one contiguous slot range.
//
// The warp finds its rows in parallel (one candidate row per lane, kept rows
// compacted by ballot into a shared list with running end offsets), then
// walks the concatenation of the rows 32 atoms at a time; a lane finds the
// row of the atom it fetches by stepping forward from the row of the round's
// first atom.  A fetched j whose distance to the bounding box of the warp's i
// atoms is not below a (cell rows overhang the cutoff sphere by up to a cell)
// is dropped there; the rest enter a 64-entry FIFO in shared memory, which is
// drained 32 at a time, so the pair loop runs full (and unrolled).  All lanes
// read each queued j by broadcast.  Per candidate a lane evaluates one rsqrt and
// 17 FP32 FMA-pipe operations (19 in the LJ pass); the FP32 passes issue all but
// the four accumulations as packed FP32x2 instructions over two queued j's (the
// FIFO then holds pair blocks x x y y z z q q, so each packed operand is one half
// of a 16-byte load).  Pairs beyond a, the pair j = i and pairs inside one rigid
// molecule get charge zero (exact zero contributions), never a branch.  More
// rows than the list holds are taken in segments.
//
// The box test computes, in the pair test's own rounding order, a lower bound
// of every r^2 the j would meet (rounding is monotone), so a dropped j is one
// that every lane would have tested out: dropping it removes exact zero
// contributions only.
//
// Each i adds its in-range j's in ascending slot order into one accumulator,
// whatever the brick shape or chunking: results are bitwise reproducible and
// independent of the launch configuration, and a system evaluated inside a
// batch (blockIdx.y = system) gives exactly the bits it gives alone.
#include "kernels.cuh"

namespace msm {

// One warp per CTA: a brick's warp frees its slot as soon as it is done (bricks
// differ in size), and 32 resident one-warp CTAs per SM at 64 registers hide the
// rsqrt and shared-load latency of the pair steps better than fewer, larger ones.
constexpr int SR_WARPS = 1;
constexpr int SR_MAXROWS = 320;     // row-list capacity per warp (a segment)

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrt_ftz(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }
template <typename T> __device__ __forceinline__ T big_t();
template <> __device__ __forceinline__ float big_t<float>() { return 1e30f; }
template <> __device__ __forceinline__ double big_t<double>() { return 1e200; }
template <typename T> __device__ __forceinline__ T inf_t();
template <> __device__ __forceinline__ float inf_t<float>() { return __int_as_float(0x7f800000); }
template <> __device__ __forceinline__ double inf_t<double>() { return __longlong_as_double(0x7ff0000000000000LL); }

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Added to every r^2 (through the FMA chain, so it costs no instruction): keeps
// rsqrt and 1/r^3 finite for the pair j = i, whose charge is masked to zero.
// Far below one ulp of any real pair distance squared, so no real pair changes.
template <typename T> __device__ __forceinline__ T r2_eps();
template <> __device__ __forceinline__ float r2_eps<float>() { return 1e-12f; }
template <> __device__ __forceinline__ double r2_eps<double>() { return 1e-30; }

template <typename T> struct ShortSmem {
    int rs0[SR_WARPS][SR_MAXROWS];      // first slot of each kept row
    int rend[SR_WARPS][SR_MAXROWS];     // running end of each row in the concatenation
    union {
        vec4<T> sj[SR_WARPS][64];       // FIFO of queued j atoms, (x, y, z, q) each
        T sp[SR_WARPS][64 * 4];         // FP32 packed passes: the same FIFO as pair blocks,
                                        // entries 2p, 2p+1 at [8p, 8p+8): x x y y z z q q
    };
    int sf[SR_WARPS][64];               // their molecule ids
};

// Two queued j's per step of the FP32 Coulomb pass, on packed FP32 pairs (one
// f32x2 instruction does the same IEEE operation for both j's).  Every per-pair
// value is computed by the operations of the scalar loop in k_short, in the same
// order (x - y as x + (-y); -poly from the negated coefficients, exact since
// rounding commutes with negation), and each accumulator takes its terms one j
// at a time in queue order: the sums are bitwise those of the scalar loop.  P
// points at pair block q0/2 of the warp's FIFO (q0 even), F at the molecule id of
// entry q0; an odd cnt reads one pad entry of charge zero beyond a of every lane.
template <bool MODEL>
__device__ __forceinline__ void pair_steps_f32x2(const float *__restrict__ P, const int *__restrict__ F,
                                                 const int cnt, const vec4<float> pi, const int mi,
                                                 const ShortArgs<float> &A, float &phi, float &ax, float &ay,
                                                 float &az)
{
    const float2 npx = make_float2(-pi.x, -pi.x), npy = make_float2(-pi.y, -pi.y), npz = make_float2(-pi.z, -pi.z);
    const float2 eps = make_float2(r2_eps<float>(), r2_eps<float>());
    const float2 nc0 = make_float2(-A.c0, -A.c0), nc1 = make_float2(-A.c1, -A.c1), nc2 = make_float2(-A.c2, -A.c2);
    const float2 d0 = make_float2(A.d0, A.d0), d1 = make_float2(A.d1, A.d1);
#pragma unroll 8
    for (int k = 0; k < cnt; k += 2) {
        const float4 xy = *reinterpret_cast<const float4 *>(P + 4 * k);
        const float4 zq = *reinterpret_cast<const float4 *>(P + 4 * k + 4);
        const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), npx);
        const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), npy);
        const float2 dz = __fadd2_rn(make_float2(zq.x, zq.y), npz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps)));
        bool in0 = r2.x < A.a2, in1 = r2.y < A.a2;
        if (MODEL) {
            const int2 f = *reinterpret_cast<const int2 *>(F + k);
            in0 = in0 & (mi != f.x);
            in1 = in1 & (mi != f.y);
        } else {
            in0 = in0 & (r2.x > 2.f * r2_eps<float>());
            in1 = in1 & (r2.y > 2.f * r2_eps<float>());
        }
        const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        const float2 ri2 = __fmul2_rn(ri, ri);
        const float2 qj = make_float2(in0 ? zq.z : 0.f, in1 ? zq.w : 0.f);
        const float2 g = __fadd2_rn(ri, __ffma2_rn(__ffma2_rn(nc2, r2, nc1), r2, nc0));     // ri - poly
        const float2 fs = __ffma2_rn(ri2, ri, __ffma2_rn(d1, r2, d0));
        const float2 sc = __fmul2_rn(qj, fs);
        phi = fmaf(qj.x, g.x, phi);
        ax = fmaf(sc.x, dx.x, ax); ay = fmaf(sc.x, dy.x, ay); az = fmaf(sc.x, dz.x, az);
        phi = fmaf(qj.y, g.y, phi);
        ax = fmaf(sc.y, dx.y, ax); ay = fmaf(sc.y, dy.y, ay); az = fmaf(sc.y, dz.y, az);
    }
}

// The same for the O-O Lennard-Jones pass (j != i by distance): sigma^2/r^2 and
// its powers, the energy difference and the force factor on packed pairs; the
// negated values the scalar loop forms by operand negation come from negated
// constants ((-s)(-s) = s s exactly, RN(-x) = -RN(x)), and le, lx, ly, lz take
// one j at a time in queue order, as in the scalar loop.
__device__ __forceinline__ void pair_steps_lj_f32x2(const float *__restrict__ P, const int cnt,
                                                    const vec4<float> pi, const ShortArgs<float> &A, float &le,
                                                    float &lx, float &ly, float &lz, int &npair)
{
    const float2 npx = make_float2(-pi.x, -pi.x), npy = make_float2(-pi.y, -pi.y), npz = make_float2(-pi.z, -pi.z);
    const float2 eps = make_float2(r2_eps<float>(), r2_eps<float>());
    const float2 ns2 = make_float2(-A.lj_s2, -A.lj_s2), two = make_float2(2.f, 2.f);
    const float2 n24 = make_float2(-A.lj_24eps, -A.lj_24eps);
#pragma unroll 8
    for (int k = 0; k < cnt; k += 2) {
        const float4 xy = *reinterpret_cast<const float4 *>(P + 4 * k);
        const float4 zq = *reinterpret_cast<const float4 *>(P + 4 * k + 4);
        const float2 dx = __fadd2_rn(make_float2(xy.x, xy.y), npx);
        const float2 dy = __fadd2_rn(make_float2(xy.z, xy.w), npy);
        const float2 dz = __fadd2_rn(make_float2(zq.x, zq.y), npz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps)));
        const bool in0 = (r2.x < A.a2) & (r2.x > 2.f * r2_eps<float>());
        const bool in1 = (r2.y < A.a2) & (r2.y > 2.f * r2_eps<float>());
        const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        const float2 ri2 = __fmul2_rn(ri, ri);
        const float2 nsr2 = __fmul2_rn(ns2, make_float2(in0 ? ri2.x : 0.f, in1 ? ri2.y : 0.f));   // -sigma^2/r^2
        const float2 nsr6 = __fmul2_rn(__fmul2_rn(nsr2, nsr2), nsr2);                           // -(sr2^3)
        const float2 sr12 = __fmul2_rn(nsr6, nsr6);
        const float2 d = __fadd2_rn(sr12, nsr6);                                               // sr12 - sr6
        const float2 nfl = __fmul2_rn(__fmul2_rn(n24, ri2), __ffma2_rn(two, sr12, nsr6));       // -fl
        le = fmaf(A.lj_4eps, d.x, le);
        npair += in0 ? 1 : 0;
        lx = fmaf(nfl.x, dx.x, lx); ly = fmaf(nfl.x, dy.x, ly); lz = fmaf(nfl.x, dz.x, lz);
        le = fmaf(A.lj_4eps, d.y, le);
        npair += in1 ? 1 : 0;
        lx = fmaf(nfl.y, dx.y, lx); ly = fmaf(nfl.y, dy.y, ly); lz = fmaf(nfl.y, dz.y, lz);
    }
}

// MODEL: rigid-water completion -- pairs inside one molecule are skipped (the
// exclusion kernel removes their smooth part); atoms that are not LJ sites get
// a zero LJ output.
// COUNT: diagnostics only -- count the pairs inside the cutoff instead of summing.
// LJP: the O-O Lennard-Jones pass of the water completion, over the LJ-site
// cell list (i and j both LJ sites, j != i, r < a), in ascending slot order;
// the constant shift of the cut-and-shifted potential is applied once per
// counted pair at the end.
// PACKED: the FP32 Coulomb and LJ passes take their queued j's two at a time on
// packed FP32 pairs (pair_steps_f32x2, pair_steps_lj_f32x2); otherwise, and for
// FP64 and the pair count, one at a time.
// WOLF: the pair term of Wolf summation (one j at a time; erfc and exp per pair).
template <typename T, bool MODEL, bool COUNT, bool LJP, bool PACKED, bool WOLF = false>
__global__ void __launch_bounds__(SR_WARPS * 32, sizeof(T) == 4 ? 32 : 16) k_short(const ShortArgs<T> A)
{
    __shared__ ShortSmem<T> S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int *BD = LJP ? D.lj_bd : D.bd, *NB = LJP ? D.lj_nb : D.nb;
    const int brick = blockIdx.x * SR_WARPS + wid;
    // i groups: warp `brick` takes group g0 + brick of this system, 32 slots
    const int *gc = A.gcol ? A.gcol + (LJP ? D.lgp_col_off : D.gp_col_off) : nullptr;
    const int g0 = gc ? gc[0] : 0;
    const int n_units = gc ? gc[LJP ? D.lgp_nc[0] * D.lgp_nc[1] : D.gp_nc[0] * D.gp_nc[1]] - g0
                           : (LJP ? D.lj_nbricks : D.nbricks);
    if (brick >= n_units || failed(A.status)) return;
    if (A.vl_ctl && A.vl_ctl[1] == 0 && A.vl_ctl[2] == 0) return;     // the Verlet-list path ran
    constexpr bool PK = PACKED && sizeof(T) == 4 && !COUNT;
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int bx = brick % NB[0], by = (brick / NB[0]) % NB[1], bz = brick / (NB[0] * NB[1]);
    const int cx0 = bx * BD[0], cx1 = min(cx0 + BD[0], nx);
    const int cy0 = by * BD[1], cy1 = min(cy0 + BD[1], ny);
    const int cz0 = bz * BD[2], cz1 = min(cz0 + BD[2], nz);
    const int *__restrict__ start = A.start + D.cell_off;
    const unsigned lt = (1u << lane) - 1u;

    int n_i = 0;
    if (gc) {
        n_i = 32;                                  // one pass over the group's (up to) 32 atoms
    } else {
        for (int cz = cz0; cz < cz1; cz++)
            for (int cy = cy0; cy < cy1; cy++) {
                const int rb = (cz * ny + cy) * nx;
                n_i += start[rb + cx1] - start[rb + cx0];
            }
    }
    const T h = (T)D.g.h, inv_h = T(1) / h;
    const T a_sel2 = A.a_sel * A.a_sel;

    for (int base = 0; base < n_i; base += 32) {
        // ---- this lane's i atom: slot lane of the group, or the (base + lane)-th atom of the brick
        int slot = -1;
        if (gc) {
            slot = A.gslot[32 * (size_t)(g0 + brick) + lane];
        } else {
            int want = base + lane, acc = 0;
            for (int cz = cz0; cz < cz1; cz++)
                for (int cy = cy0; cy < cy1; cy++) {
                    const int rb = (cz * ny + cy) * nx;
                    const int s0 = start[rb + cx0], c = start[rb + cx1] - s0;
                    if (slot < 0 && want < acc + c) slot = s0 + (want - acc);
                    acc += c;
                }
        }
        const bool valid = slot >= 0;
        const vec4<T> pi = valid ? A.apos[slot] : vec4<T>{big_t<T>(), big_t<T>(), big_t<T>(), T(0)};
        const int mi = (MODEL && valid) ? A.aflag[slot] >> 1 : -1;     // molecule id (-1: no i atom)

        // ---- bounding box of the valid i atoms
        T lo[3], hi[3];
        lo[0] = warp_min(valid ? pi.x : inf_t<T>()); hi[0] = warp_max(valid ? pi.x : -inf_t<T>());
        lo[1] = warp_min(valid ? pi.y : inf_t<T>()); hi[1] = warp_max(valid ? pi.y : -inf_t<T>());
        lo[2] = warp_min(valid ? pi.z : inf_t<T>()); hi[2] = warp_max(valid ? pi.z : -inf_t<T>());

        T phi = 0, ax = 0, ay = 0, az = 0;
        T lx = 0, ly = 0, lz = 0, le = 0;
        int npair = 0;
        int head = 0, npend = 0;        // FIFO: queued j's at [head, head + npend) mod 64, head in {0, 32}

        // sum the cnt queued j's from FIFO position q0 (no wrap: q0 + cnt <= 64)
        auto pairs = [&](const int q0, const int cnt) {
#pragma unroll (LJP ? 8 : 32)
            for (int k = 0; k < cnt; k++) {
                const vec4<T> pj = S.sj[wid][q0 + k];
                const T dx = pj.x - pi.x, dyy = pj.y - pi.y, dzz = pj.z - pi.z;
                const T r2s = fma(dx, dx, fma(dyy, dyy, fma(dzz, dzz, r2_eps<T>())));
                bool in = r2s < A.a2;
                // j = i: the water model's molecule test excludes it (an atom is in its own
                // molecule); bare charges and the LJ pass (whose sites are one per molecule)
                // test the distance
                if (MODEL) in = in & (mi != S.sf[wid][q0 + k]);
                else in = in & (r2s > T(2) * r2_eps<T>());
                if (COUNT) { npair += in ? 1 : 0; continue; }
                const T ri = rsqrt_t<T>(r2s);
                const T ri2 = ri * ri;
                if (LJP) {
                    // masked pairs get sigma^2/r^2 = 0, so every term vanishes; the shift of
                    // the cut-and-shifted potential is applied once per counted pair at the end
                    const T sr2 = A.lj_s2 * (in ? ri2 : T(0));
                    const T sr6 = sr2 * sr2 * sr2, sr12 = sr6 * sr6;
                    le = fma(A.lj_4eps, sr12 - sr6, le);
                    npair += in ? 1 : 0;
                    const T fl = (A.lj_24eps * ri2) * fma(T(2), sr12, -sr6);
                    lx = fma(-fl, dx, lx); ly = fma(-fl, dyy, ly); lz = fma(-fl, dzz, lz);
                    continue;
                }
                const T qj = in ? pj.w : T(0);
                T g, fs;                 // pair term and -g'(r)/r
                if constexpr (WOLF) {
                    const T ar = A.w_alpha * (r2s * ri);
                    const T ec = erfc(ar);
                    const T ex = exp(-ar * ar);
                    g = fma(ec, ri, -A.w_shift);
                    fs = fma(ec, ri, A.w_c * ex) * ri2;
                } else {
                    const T poly = fma(fma(A.c2, r2s, A.c1), r2s, A.c0);
                    g = ri - poly;
                    fs = fma(ri2, ri, fma(A.d1, r2s, A.d0));
                }
                phi = fma(qj, g, phi);
                const T sc = qj * fs;
                ax = fma(sc, dx, ax); ay = fma(sc, dyy, ay); az = fma(sc, dzz, az);
            }
        };

        const int zlo = max(0, (int)floor((lo[2] - A.a_sel) * inv_h));
        const int zhi = min(nz - 1, (int)floor((hi[2] + A.a_sel) * inv_h));
        const int ylo = max(0, (int)floor((lo[1] - A.a_sel) * inv_h));
        const int yhi = min(ny - 1, (int)floor((hi[1] + A.a_sel) * inv_h));
        const int nyr = yhi - ylo + 1, nr_all = max(0, zhi - zlo + 1) * max(0, nyr);
        int r_next = 0;
        while (r_next < nr_all) {
            // ---- a segment of kept rows, in (z, y) order
            int nrows = 0, total = 0;
            while (r_next < nr_all) {
                const int r = r_next + lane;
                int s0 = 0, len = 0;
                if (r < nr_all) {
                    const int cz = zlo + r / nyr, cy = ylo + r % nyr;
                    const T dz = max(T(0), max(T(cz) * h - hi[2], lo[2] - T(cz + 1) * h));
                    const T dy = max(T(0), max(T(cy) * h - hi[1], lo[1] - T(cy + 1) * h));
                    const T dyz2 = dy * dy + dz * dz;
                    if (dyz2 < a_sel2) {
                        const T rx = sqrt(a_sel2 - dyz2);
                        const int xlo = max(0, (int)floor((lo[0] - rx) * inv_h));
                        const int xhi = min(nx - 1, (int)floor((hi[0] + rx) * inv_h));
                        if (xlo <= xhi) {
                            const int rb = (cz * ny + cy) * nx;
                            s0 = start[rb + xlo];
                            len = start[rb + xhi + 1] - s0;
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, len > 0);
                if (nrows + __popc(m) > SR_MAXROWS) break;           // uniform: flush this segment first
                int incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (len > 0) {
                    const int pos = nrows + __popc(m & lt);
                    S.rs0[wid][pos] = s0;
                    S.rend[wid][pos] = total + incl;
                }
                nrows += __popc(m);
                total += __shfl_sync(0xffffffffu, incl, 31);
                r_next += 32;
            }
            __syncwarp();
            // ---- fetch the segment's atoms 32 at a time, queue those near the box.  The
            // rows are consumed in order: rc is the row holding atom cb of the concatenation,
            // and a lane steps forward from it to the row holding its own atom.
            int rc = 0;
            for (int cb = 0; cb < total; cb += 32) {
                const int cnt = min(32, total - cb);
                bool keep = false;
                vec4<T> pj{T(0), T(0), T(0), T(0)};
                int fj = 0, row = rc;
                if (lane < cnt) {
                    const int want = cb + lane;
                    while (S.rend[wid][row] <= want) row++;
                    const int js = S.rs0[wid][row] + (want - (row ? S.rend[wid][row - 1] : 0));
                    pj = A.apos[js];
                    if (MODEL) fj = A.aflag[js] >> 1;              // molecule id
                    const T ex = max(T(0), max(lo[0] - pj.x, pj.x - hi[0]));
                    const T ey = max(T(0), max(lo[1] - pj.y, pj.y - hi[1]));
                    const T ez = max(T(0), max(lo[2] - pj.z, pj.z - hi[2]));
                    keep = fma(ex, ex, fma(ey, ey, fma(ez, ez, r2_eps<T>()))) < A.a2;
                }
                rc = __shfl_sync(0xffffffffu, row, 31);             // row of atom cb + 31
                if (cnt == 32 && rc < nrows - 1 && S.rend[wid][rc] <= cb + 32) rc++;
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int q = (head + npend + __popc(m & lt)) & 63;
                    if constexpr (PK) {
                        T *e = &S.sp[wid][8 * (q >> 1) + (q & 1)];
                        e[0] = pj.x; e[2] = pj.y; e[4] = pj.z; e[6] = pj.w;
                    } else {
                        S.sj[wid][q] = pj;
                    }
                    if (MODEL) S.sf[wid][q] = fj;
                }
                npend += __popc(m);
                __syncwarp();
                if (npend >= 32) {
                    if constexpr (PK && LJP)
                        pair_steps_lj_f32x2(&S.sp[wid][4 * head], 32, pi, A, le, lx, ly, lz, npair);
                    else if constexpr (PK)
                        pair_steps_f32x2<MODEL>(&S.sp[wid][4 * head], &S.sf[wid][head], 32, pi, mi, A, phi, ax, ay, az);
                    else
                        pairs(head, 32);
                    head ^= 32;
                    npend -= 32;
                    __syncwarp();
                }
            }
        }
        if (npend > 0) {
            if constexpr (PK) {
                if ((npend & 1) && lane == 0) {
                    // pad entry: charge zero, 2a beyond the box in x (out of range of every
                    // lane, finite distances: exact zero terms in both passes)
                    T *e = &S.sp[wid][8 * ((head + npend) >> 1) + 1];
                    e[0] = lo[0] - T(2) * A.a; e[2] = T(0.5) * (lo[1] + hi[1]);
                    e[4] = T(0.5) * (lo[2] + hi[2]); e[6] = T(0);
                    S.sf[wid][head + npend] = -2;
                }
                __syncwarp();
                if constexpr (LJP)
                    pair_steps_lj_f32x2(&S.sp[wid][4 * head], npend, pi, A, le, lx, ly, lz, npair);
                else
                    pair_steps_f32x2<MODEL>(&S.sp[wid][4 * head], &S.sf[wid][head], npend, pi, mi, A, phi, ax, ay, az);
            } else {
                pairs(head, npend);
            }
            __syncwarp();
        }
        if (valid) {
            if (COUNT) { A.cnt[slot] = (double)npair; continue; }
            const int atom = A.perm[slot];
            if (LJP) { A.lj[atom] = vec4<T>{lx, ly, lz, fma(-A.lj_shift, (T)npair, le)}; continue; }
            A.sr[atom] = vec4<T>{-pi.w * ax, -pi.w * ay, -pi.w * az, phi};
            if (MODEL && !(A.aflag[slot] & 1)) A.lj[atom] = vec4<T>{T(0), T(0), T(0), T(0)};
        }
    }
}

// ------------------------------------------------------------- i groups

// One warp per column of cw x cw cells: its atom count over all cell layers, as
// whole groups of 32.
template <bool LJ>
__global__ void __launch_bounds__(128) k_grp_count(const Batch bt, const int *__restrict__ start,
                                                   int *__restrict__ gcnt, const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int cw = LJ ? D.lgp_cw : D.gp_cw, ncx = LJ ? D.lgp_nc[0] : D.gp_nc[0], ncy = LJ ? D.lgp_nc[1] : D.gp_nc[1];
    const int col = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (col >= ncx * ncy || failed(status)) return;
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int cx0 = (col % ncx) * cw, cx1 = min(cx0 + cw, nx), cy0 = (col / ncx) * cw, cy1 = min(cy0 + cw, ny);
    const int *__restrict__ st = start + D.cell_off;
    int c = 0;
    for (int cz = lane; cz < nz; cz += 32)
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            c += st[rb + cx1] - st[rb + cx0];
        }
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) gcnt[(LJ ? D.lgp_col_off : D.gp_col_off) + col] = (c + 31) / 32;
}

// One warp per (column, chunk of 32 cell layers), lane = layer: the slots of the
// column's atoms, layer by layer, each layer's atoms in ascending z (ties by
// slot), into its groups, -1 after the last atom.  Ordering by z inside a layer
// gives the groups that cut a layer thinner boxes.  A lane loads its layer's z
// values into its own column of shared memory (entry e of lane l at [e][l]: no
// bank is shared) and sorts them there by insertion; a layer of more than
// GF_MAXL atoms keeps the cell order (the grouping changes no result).
constexpr int GF_MAXL = 24;
template <typename T, bool LJ>
__global__ void __launch_bounds__(128) k_grp_fill(const Batch bt, const int *__restrict__ start,
                                                  const vec4<T> *__restrict__ apos, const int *__restrict__ gcol,
                                                  int *__restrict__ gslot, const int *__restrict__ status)
{
    __shared__ float skey[4][GF_MAXL][32];
    __shared__ int sslot[4][GF_MAXL][32];
    const SysDesc &D = bt.sd[blockIdx.y];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cw = LJ ? D.lgp_cw : D.gp_cw, ncx = LJ ? D.lgp_nc[0] : D.gp_nc[0], ncy = LJ ? D.lgp_nc[1] : D.gp_nc[1];
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int nchunk = (nz + 31) / 32;
    const int idx = blockIdx.x * 4 + w, col = idx / nchunk, z0 = 32 * (idx % nchunk);
    if (col >= ncx * ncy || failed(status)) return;
    const int cx0 = (col % ncx) * cw, cx1 = min(cx0 + cw, nx), cy0 = (col / ncx) * cw, cy1 = min(cy0 + cw, ny);
    const int *__restrict__ st = start + D.cell_off;
    const int gcl = (LJ ? D.lgp_col_off : D.gp_col_off) + col;
    int *out = gslot + 32 * (size_t)gcol[gcl];
    auto layer_count = [&](int cz) {
        int c = 0;
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            c += st[rb + cx1] - st[rb + cx0];
        }
        return c;
    };
    // atoms of the column below this chunk
    int below = 0;
    for (int cz = lane; cz < z0; cz += 32) below += layer_count(cz);
#pragma unroll
    for (int o = 16; o; o >>= 1) below += __shfl_xor_sync(0xffffffffu, below, o);
    const int cz = z0 + lane;
    const int c = cz < nz ? layer_count(cz) : 0;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    int r = below + incl - c;
    if (c > 0 && c <= GF_MAXL) {
        int n = 0;
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            const int s0 = st[rb + cx0], s1 = st[rb + cx1];
            // four position loads in flight at a time
#pragma unroll 4
            for (int s = s0; s < s1; s++) {
                skey[w][n + (s - s0)][lane] = (float)apos[s].z;
                sslot[w][n + (s - s0)][lane] = s;
            }
            n += s1 - s0;
        }
        // insertion by (z, slot): slots were loaded in ascending order, so ties stay in order
        for (int e = 1; e < n; e++) {
            const float zk = skey[w][e][lane];
            const int sk = sslot[w][e][lane];
            int k = e;
            while (k > 0 && skey[w][k - 1][lane] > zk) {
                skey[w][k][lane] = skey[w][k - 1][lane];
                sslot[w][k][lane] = sslot[w][k - 1][lane];
                k--;
            }
            skey[w][k][lane] = zk;
            sslot[w][k][lane] = sk;
        }
        for (int e = 0; e < n; e++) out[r++] = sslot[w][e][lane];
    } else if (c > 0) {
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            for (int s = st[rb + cx0]; s < st[rb + cx1]; s++) out[r++] = s;
        }
    }
    if (z0 + 32 >= nz) {                       // the column's last chunk pads its last group
        const int total = below + __shfl_sync(0xffffffffu, incl, 31);
        const int ntot = 32 * (gcol[gcl + 1] - gcol[gcl]);
        for (int q = total + lane; q < ntot; q += 32) out[q] = -1;
    }
}

template <typename T>
int launch_groups(const Batch &bt, bool lj, int max_cols, int max_nz, int n_cols, const int *start,
                  const vec4<T> *apos, int *gcnt, int *gcol, int *bsum, int *gslot, const int *status, cudaStream_t st)
{
    if (max_cols <= 0) return MSM_OK;
    const dim3 grid((max_cols + 3) / 4, bt.B);
    if (lj) k_grp_count<true><<<grid, 128, 0, st>>>(bt, start, gcnt, status);
    else k_grp_count<false><<<grid, 128, 0, st>>>(bt, start, gcnt, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    const int rc = launch_scan(n_cols, gcnt, gcol, bsum, status, st);
    if (rc != MSM_OK) return rc;
    // fill: one warp per (column, chunk of 32 layers)
    const dim3 gfill((max_cols * ((max_nz + 31) / 32) + 3) / 4, bt.B);
    if (lj) k_grp_fill<T, true><<<gfill, 128, 0, st>>>(bt, start, apos, gcol, gslot, status);
    else k_grp_fill<T, false><<<gfill, 128, 0, st>>>(bt, start, apos, gcol, gslot, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_short(const ShortArgs<T> &a, bool model, cudaStream_t st)
{
    if (a.max_bricks <= 0) return MSM_OK;
    const dim3 grid((a.max_bricks + SR_WARPS - 1) / SR_WARPS, a.bt.B);
    if (a.wolf) {
        if (model) k_short<T, true, false, false, false, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
        else k_short<T, false, false, false, false, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
        count_launch();
        CUDA_TRY(cudaGetLastError());
        return MSM_OK;
    }
    bool packed = false;
    if constexpr (sizeof(T) == 4) packed = !a.scalar_pairs;
    if constexpr (sizeof(T) == 4) {
        if (packed) {
            if (model) k_short<T, true, false, false, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
            else k_short<T, false, false, false, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
        }
    }
    if (!packed) {
        if (model) k_short<T, true, false, false, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
        else k_short<T, false, false, false, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    }
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_short_lj(const ShortArgs<T> &a, cudaStream_t st)
{
    if (a.max_bricks <= 0) return MSM_OK;
    const dim3 grid((a.max_bricks + SR_WARPS - 1) / SR_WARPS, a.bt.B);
    bool packed = false;
    if constexpr (sizeof(T) == 4) {
        packed = !a.scalar_pairs;
        if (packed) k_short<T, false, false, true, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
    }
    if (!packed) k_short<T, false, false, true, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_count_pairs(const ShortArgs<T> &a, cudaStream_t st)
{
    if (a.max_bricks <= 0) return MSM_OK;
    const dim3 grid((a.max_bricks + SR_WARPS - 1) / SR_WARPS, a.bt.B);
    k_short<T, false, true, false, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ------------------------------------------------------ LJ-site cell list

__global__ void k_lj_count(int m, const int *__restrict__ start, const int *__restrict__ aflag,
                           int *__restrict__ lj_count, const int *__restrict__ status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m || failed(status)) return;
    int k = 0;
    for (int s = start[c]; s < start[c + 1]; s++) k += aflag[s] & 1;
    lj_count[c] = k;
}

template <typename T>
__global__ void k_lj_compact(int m, const int *__restrict__ start, const int *__restrict__ lj_start,
                             const vec4<T> *__restrict__ apos, const int *__restrict__ aflag,
                             const int *__restrict__ perm, vec4<T> *__restrict__ lj_apos, int *__restrict__ lj_flag,
                             int *__restrict__ lj_perm, const int *__restrict__ status)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m || failed(status)) return;
    int k = lj_start[c];
    for (int s = start[c]; s < start[c + 1]; s++) {
        const int f = aflag[s];
        if (!(f & 1)) continue;
        lj_apos[k] = apos[s];
        lj_flag[k] = f;
        lj_perm[k] = perm[s];
        k++;
    }
}

template <typename T>
int launch_lj_count(int m_total, const int *start, const int *aflag, int *lj_count, const int *status,
                    cudaStream_t st)
{
    if (m_total <= 0) return MSM_OK;
    k_lj_count<<<(m_total + 255) / 256, 256, 0, st>>>(m_total, start, aflag, lj_count, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_lj_compact(int m_total, const int *start, const int *lj_start, const vec4<T> *apos, const int *aflag,
                      const int *perm, vec4<T> *lj_apos, int *lj_flag, int *lj_perm, const int *status,
                      cudaStream_t st)
{
    if (m_total <= 0) return MSM_OK;
    k_lj_compact<T><<<(m_total + 255) / 256, 256, 0, st>>>(m_total, start, lj_start, apos, aflag, perm, lj_apos,
                                                           lj_flag, lj_perm, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_groups<float>(const Batch &, bool, int, int, int, const int *, const vec4<float> *, int *,
                                  int *, int *, int *, const int *, cudaStream_t);
template int launch_groups<double>(const Batch &, bool, int, int, int, const int *, const vec4<double> *, int *,
                                   int *, int *, int *, const int *, cudaStream_t);
template int launch_short<float>(const ShortArgs<float> &, bool, cudaStream_t);
template int launch_short<double>(const ShortArgs<double> &, bool, cudaStream_t);
template int launch_count_pairs<float>(const ShortArgs<float> &, cudaStream_t);
template int launch_count_pairs<double>(const ShortArgs<double> &, cudaStream_t);
template int launch_short_lj<float>(const ShortArgs<float> &, cudaStream_t);
template int launch_short_lj<double>(const ShortArgs<double> &, cudaStream_t);
template int launch_lj_count<float>(int, const int *, const int *, int *, const int *, cudaStream_t);
template int launch_lj_count<double>(int, const int *, const int *, int *, const int *, cudaStream_t);
template int launch_lj_compact<float>(int, const int *, const int *, const vec4<float> *, const int *, const int *,
                                      vec4<float> *, int *, int *, const int *, cudaStream_t);
template int launch_lj_compact<double>(int, const int *, const int *, const vec4<double> *, const int *, const int *,
                                       vec4<double> *, int *, int *, const int *, cudaStream_t);

}  // namespace msm
