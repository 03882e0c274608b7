// k_cluster.cu -- the short-range part of the MSM (Sec. 3, step 1) on cluster
// pairs, FP32:
//   u_i^short = sum_{j != i, r_ij < a} q_j g*(r_ij),
//   F_i^short = q_i sum_j q_j [1/r^3 - 5/(2a^3) + 3r^2/(2a^5)] (r_i - r_j),
// the same sums as k_short.cu (and its simple-cutoff instance, g = 1/r), in a
// layout with fewer pair evaluations per pair within a.
//
// Clusters.  The finest cells are grouped into columns of 2 x 2 cells in (x, y).
// A column's atoms, taken in the order of the cell sort (z, then y, then x,
// then slot), are cut into i clusters of 8 atoms, each split into two j
// clusters of 4; the last i cluster of a column is padded with entries of
// charge zero far outside every box.  Every j cluster keeps its bounding box.
// k_cp_count counts each column's atoms per cell layer z (a prefix table, so
// the clusters that hold the atoms of layers z0..z1 are found in O(1)); a scan
// gives each column's first cluster; k_cp_fill copies the atoms (position and
// charge, molecule id, slot) into cluster order and writes the boxes.
//
// Pairs.  One warp owns one i cluster: lane = (i, js), i = lane % 8 the i atom,
// js = lane / 8 the j slot.  The warp lists the columns whose (x, y) extent
// lies within a of its box, and for each the run of clusters covering the cell
// layers within reach (one candidate column per lane, runs compacted by
// ballot), then walks the runs 32 clusters at a time, one per lane: a cluster
// whose box lies at least a from the i cluster's box is dropped, the atoms of
// the rest are loaded by groups of four lanes (eight clusters per load) into a
// 64-cluster FIFO in shared memory, drained 8 at a time.  In a drain, lane
// (i, js) takes atom js of each queued cluster, two clusters per packed FP32x2
// step (the operations of k_short's packed pair step).  Pairs beyond a, the
// pair j = i and pairs inside one rigid molecule get charge zero, never a
// branch.  At the end the four j slots of each i atom are added by two
// butterfly shuffles.
//
// Both culls compute lower bounds of the pair test's own r^2 in its rounding
// order (rounding is monotone), so only exact zero contributions are dropped.
// Each i atom sums its terms in a fixed order (runs, then clusters, per j slot;
// the slots by the butterfly), whatever the launch: results are bitwise
// reproducible, and a system inside a batch (blockIdx.y) gives the bits it
// gives alone.  The order differs from k_short's, so the two paths agree to
// rounding, not bitwise.
#include "kernels.cuh"

namespace msm {

constexpr int CP_MAXRUNS = 64;      // run-list capacity per warp (a segment)
constexpr float CP_PAD = -1000.f;   // position of padding entries (nm, relative to the box origin)
constexpr int CP_SP = 34, CP_SF = 10;   // FIFO strides of a pair block (floats, ints)

// ---------------------------------------------------------------- columns

// One warp per column: atoms of the column in each cell layer z, as the
// exclusive prefix zc[z] (z = 0..nz), and the column's clusters of 4 (a whole
// number of i clusters of 8).
__global__ void __launch_bounds__(128) k_cp_count(const Batch bt, const int *__restrict__ start, int *__restrict__ zc,
                                                  int *__restrict__ col_n, const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (col >= D.cp_nc[0] * D.cp_nc[1] || failed(status)) return;
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int px = col % D.cp_nc[0], py = col / D.cp_nc[0];
    const int cx0 = 2 * px, cx1 = min(cx0 + 2, nx), cy0 = 2 * py, cy1 = min(cy0 + 2, ny);
    const int *__restrict__ st = start + D.cell_off;
    int *z = zc + D.zc_off + (size_t)col * (nz + 1);
    int carry = 0;
    for (int z0 = 0; z0 < nz; z0 += 32) {
        const int cz = z0 + lane;
        int c = 0;
        if (cz < nz)
            for (int cy = cy0; cy < cy1; cy++) {
                const int rb = (cz * ny + cy) * nx;
                c += st[rb + cx1] - st[rb + cx0];
            }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (cz < nz) z[cz] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        z[nz] = carry;
        col_n[D.col_off + col] = ((carry + 7) / 8) * 2;
    }
}

// One warp per column: the column's atoms into cluster order (lane = cell
// layer), padding up to whole i clusters, then the box of each cluster of 4
// (lane = cluster).  An empty cluster gets the box (+inf, -inf): no box test
// passes it.
template <bool MODEL>
__global__ void __launch_bounds__(128) k_cp_fill(const ClusterArgs A)
{
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int col = blockIdx.x * 4 + (threadIdx.x >> 5);
    if (col >= D.cp_nc[0] * D.cp_nc[1] || failed(A.status)) return;
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int px = col % D.cp_nc[0], py = col / D.cp_nc[0];
    const int cx0 = 2 * px, cx1 = min(cx0 + 2, nx), cy0 = 2 * py, cy1 = min(cy0 + 2, ny);
    const int *__restrict__ st = A.start + D.cell_off;
    const int *z = A.zc + D.zc_off + (size_t)col * (nz + 1);
    const int c4 = A.col_cl[D.col_off + col], n = z[nz], npad = ((n + 7) / 8) * 8;
    const size_t e0 = 4 * (size_t)c4;
    for (int z0 = 0; z0 < nz; z0 += 32) {
        const int cz = z0 + lane;
        if (cz >= nz) continue;
        int r = z[cz];
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            for (int s = st[rb + cx0]; s < st[rb + cx1]; s++, r++) {
                A.cpos[e0 + r] = A.apos[s];
                A.cmol[e0 + r] = MODEL ? A.aflag[s] >> 1 : 0;
                A.cslot[e0 + r] = s;
            }
        }
    }
    for (int r = n + lane; r < npad; r += 32) {
        A.cpos[e0 + r] = vec4<float>{CP_PAD, CP_PAD, CP_PAD, 0.f};
        A.cmol[e0 + r] = -2;
        A.cslot[e0 + r] = -1;
    }
    __syncwarp();
    const float inf = __int_as_float(0x7f800000);
    for (int k = lane; k < npad / 4; k += 32) {
        vec4<float> lo{inf, inf, inf, 0.f}, hi{-inf, -inf, -inf, 0.f};
        for (int e = 0; e < 4; e++) {
            const size_t ee = e0 + 4 * (size_t)k + e;
            if (A.cslot[ee] < 0) continue;
            const vec4<float> p = A.cpos[ee];
            lo.x = fminf(lo.x, p.x); lo.y = fminf(lo.y, p.y); lo.z = fminf(lo.z, p.z);
            hi.x = fmaxf(hi.x, p.x); hi.y = fmaxf(hi.y, p.y); hi.z = fmaxf(hi.z, p.z);
        }
        A.cbox[2 * ((size_t)c4 + k)] = lo;
        A.cbox[2 * ((size_t)c4 + k) + 1] = hi;
    }
}

// ---------------------------------------------------------------- pairs

struct CpSmem {
    int rs0[CP_MAXRUNS];            // first cluster of each kept run
    int rend[CP_MAXRUNS];           // running end of each run in the concatenation
    // FIFO of 64 clusters as 32 pair blocks: clusters 2p, 2p+1 at [CP_SP p, CP_SP p + 32),
    // atom js at +8 js: x x y y z z q q; molecule ids of atom js at CP_SF p + 2 js.  Over
    // 16 consecutive pair blocks the strides (34 and 10 words) give 16 distinct even
    // bank offsets, so the 32 lanes storing 32 consecutive clusters hit 32 banks.
    float sp[32 * CP_SP];
    int sf[32 * CP_SF];
    int kj[32];                     // this round's kept clusters, in order
};

// npair pair blocks from P (stride CP_SP floats) and F (stride CP_SF ints) for
// the lane's j slot: two clusters per step on packed FP32 pairs, the operations
// and order of k_short's packed Coulomb step.
template <bool MODEL>
__device__ __forceinline__ void cp_steps(const float *__restrict__ P, const int *__restrict__ F, const int npair,
                                         const vec4<float> pi, const int mi, const ClusterArgs &A,
                                         float &phi, float &ax, float &ay, float &az)
{
    const float2 npx = make_float2(-pi.x, -pi.x), npy = make_float2(-pi.y, -pi.y), npz = make_float2(-pi.z, -pi.z);
    const float2 eps = make_float2(1e-12f, 1e-12f);
    const float2 nc0 = make_float2(-A.c0, -A.c0), nc1 = make_float2(-A.c1, -A.c1), nc2 = make_float2(-A.c2, -A.c2);
    const float2 d0 = make_float2(A.d0, A.d0), d1 = make_float2(A.d1, A.d1);
#pragma unroll 4
    for (int p = 0; p < npair; p++) {
        const float2 xx = *reinterpret_cast<const float2 *>(P + CP_SP * p);
        const float2 yy = *reinterpret_cast<const float2 *>(P + CP_SP * p + 2);
        const float2 zz = *reinterpret_cast<const float2 *>(P + CP_SP * p + 4);
        const float2 qq = *reinterpret_cast<const float2 *>(P + CP_SP * p + 6);
        const float2 dx = __fadd2_rn(xx, npx);
        const float2 dy = __fadd2_rn(yy, npy);
        const float2 dz = __fadd2_rn(zz, npz);
        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps)));
        bool in0 = r2.x < A.a2, in1 = r2.y < A.a2;
        if (MODEL) {
            const int2 f = *reinterpret_cast<const int2 *>(F + CP_SF * p);
            in0 = in0 & (mi != f.x);
            in1 = in1 & (mi != f.y);
        } else {
            in0 = in0 & (r2.x > 2e-12f);
            in1 = in1 & (r2.y > 2e-12f);
        }
        const float2 ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
        const float2 ri2 = __fmul2_rn(ri, ri);
        const float2 qj = make_float2(in0 ? qq.x : 0.f, in1 ? qq.y : 0.f);
        const float2 g = __fadd2_rn(ri, __ffma2_rn(__ffma2_rn(nc2, r2, nc1), r2, nc0));     // ri - poly
        const float2 fs = __ffma2_rn(ri2, ri, __ffma2_rn(d1, r2, d0));
        const float2 sc = __fmul2_rn(qj, fs);
        phi = fmaf(qj.x, g.x, phi);
        ax = fmaf(sc.x, dx.x, ax); ay = fmaf(sc.x, dy.x, ay); az = fmaf(sc.x, dz.x, az);
        phi = fmaf(qj.y, g.y, phi);
        ax = fmaf(sc.y, dx.y, ax); ay = fmaf(sc.y, dy.y, ay); az = fmaf(sc.y, dz.y, az);
    }
}

template <bool MODEL>
__global__ void __launch_bounds__(32, 32) k_cp_short(const ClusterArgs A)
{
    __shared__ __align__(16) CpSmem S;
    const int lane = threadIdx.x;
    const SysDesc &D = A.bt.sd[blockIdx.y];
    if (failed(A.status)) return;
    if (A.vl_ctl && A.vl_ctl[1] == 0 && A.vl_ctl[2] == 0) return;     // the Verlet-list path ran
    const int ncx = D.cp_nc[0], ncy = D.cp_nc[1];
    const int c0 = A.col_cl[D.col_off], c1 = A.col_cl[D.col_off + ncx * ncy];
    if (2 * (int)blockIdx.x >= c1 - c0) return;
    const int I = c0 / 2 + blockIdx.x;                 // this warp's i cluster (global, units of 8)
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const unsigned lt = (1u << lane) - 1u;

    const int ii = lane & 7, js = lane >> 3;
    const size_t ei = 8 * (size_t)I + ii;
    const vec4<float> pi = A.cpos[ei];
    const int slot = A.cslot[ei];
    const bool valid = slot >= 0;
    const int mi = (MODEL && valid) ? A.cmol[ei] : -1;
    // box of the i cluster: the union of its two clusters of 4
    float lo[3], hi[3];
    {
        const vec4<float> l0 = A.cbox[4 * (size_t)I], h0 = A.cbox[4 * (size_t)I + 1];
        const vec4<float> l1 = A.cbox[4 * (size_t)I + 2], h1 = A.cbox[4 * (size_t)I + 3];
        lo[0] = fminf(l0.x, l1.x); lo[1] = fminf(l0.y, l1.y); lo[2] = fminf(l0.z, l1.z);
        hi[0] = fmaxf(h0.x, h1.x); hi[1] = fmaxf(h0.y, h1.y); hi[2] = fmaxf(h0.z, h1.z);
    }
    const float h = (float)D.g.h, inv_h = 1.f / h, inv_2h = 0.5f * inv_h;
    const float a_sel = A.a_sel, a_sel2 = a_sel * a_sel;
    const int pxlo = max(0, (int)floorf((lo[0] - a_sel) * inv_2h)), pxhi = min(ncx - 1, (int)floorf((hi[0] + a_sel) * inv_2h));
    const int pylo = max(0, (int)floorf((lo[1] - a_sel) * inv_2h)), pyhi = min(ncy - 1, (int)floorf((hi[1] + a_sel) * inv_2h));
    const int nrx = pxhi - pxlo + 1, nall = max(0, nrx) * max(0, pyhi - pylo + 1);
    const int *zcs = A.zc + D.zc_off;

    float phi = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
    int head = 0, npend = 0;            // FIFO: queued clusters at [head, head + npend) mod 64, head % 8 == 0
    int r_next = 0;
    while (r_next < nall) {
        // ---- a segment of kept runs, in (py, px) order
        int nruns = 0, total = 0;
        while (r_next < nall) {
            const int r = r_next + lane;
            int s0 = 0, len = 0;
            if (r < nall) {
                const int px = pxlo + r % nrx, py = pylo + r / nrx;
                const int cx1 = min(2 * px + 2, nx), cy1 = min(2 * py + 2, ny);
                const float ex = fmaxf(0.f, fmaxf((float)(2 * px) * h - hi[0], lo[0] - (float)cx1 * h));
                const float ey = fmaxf(0.f, fmaxf((float)(2 * py) * h - hi[1], lo[1] - (float)cy1 * h));
                const float dxy2 = ex * ex + ey * ey;
                if (dxy2 < a_sel2) {
                    const float rz = sqrtf(a_sel2 - dxy2);
                    const int zlo = max(0, (int)floorf((lo[2] - rz) * inv_h));
                    const int zhi = min(nz - 1, (int)floorf((hi[2] + rz) * inv_h));
                    if (zlo <= zhi) {
                        const int col = py * ncx + px;
                        const int *z = zcs + (size_t)col * (nz + 1);
                        const int cb = A.col_cl[D.col_off + col];
                        s0 = cb + z[zlo] / 4;
                        len = cb + (z[zhi + 1] + 3) / 4 - s0;
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, len > 0);
            if (nruns + __popc(m) > CP_MAXRUNS) break;           // uniform: flush this segment first
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (len > 0) {
                const int pos = nruns + __popc(m & lt);
                S.rs0[pos] = s0;
                S.rend[pos] = total + incl;
            }
            nruns += __popc(m);
            total += __shfl_sync(0xffffffffu, incl, 31);
            r_next += 32;
        }
        __syncwarp();
        // ---- the segment's clusters 32 at a time, one per lane for the box test; the
        // atoms of the kept clusters are then loaded by groups of four lanes, eight
        // clusters per load instruction (runs are contiguous: few cache lines per load)
        int rc = 0;
        for (int cb = 0; cb < total; cb += 32) {
            const int want = cb + lane;
            bool keep = false;
            int J = 0, row = rc;
            if (want < total) {
                while (S.rend[row] <= want) row++;
                J = S.rs0[row] + (want - (row ? S.rend[row - 1] : 0));
                const vec4<float> jl = A.cbox[2 * (size_t)J], jh = A.cbox[2 * (size_t)J + 1];
                const float ex = fmaxf(0.f, fmaxf(jl.x - hi[0], lo[0] - jh.x));
                const float ey = fmaxf(0.f, fmaxf(jl.y - hi[1], lo[1] - jh.y));
                const float ez = fmaxf(0.f, fmaxf(jl.z - hi[2], lo[2] - jh.z));
                keep = fmaf(ex, ex, fmaf(ey, ey, fmaf(ez, ez, 1e-12f))) < A.a2;
            }
            rc = __shfl_sync(0xffffffffu, row, 31);             // run of cluster cb + 31
            if (rc < nruns - 1 && S.rend[rc] <= cb + 32) rc++;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            const int nk = __popc(m);
            if (keep) S.kj[__popc(m & lt)] = J;
            __syncwarp();
            // kept cluster r = 8 t + lane / 4, atom lane % 4, for t = 0..3: all loads first
            float4 pj[4];
            int fj[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int r = 8 * t + (lane >> 2);
                if (r < nk) {
                    const size_t e = 4 * (size_t)S.kj[r] + (lane & 3);
                    pj[t] = *reinterpret_cast<const float4 *>(A.cpos + e);
                    fj[t] = MODEL ? A.cmol[e] : 0;
                }
            }
#pragma unroll
            for (int t = 0; t < 4; t++) {
                const int r = 8 * t + (lane >> 2);
                if (r < nk) {
                    const int q = (head + npend + r) & 63, k = lane & 3;
                    float *e = &S.sp[CP_SP * (q >> 1) + 8 * k + (q & 1)];
                    e[0] = pj[t].x; e[2] = pj[t].y; e[4] = pj[t].z; e[6] = pj[t].w;
                    if (MODEL) S.sf[CP_SF * (q >> 1) + 2 * k + (q & 1)] = fj[t];
                }
            }
            npend += nk;
            __syncwarp();
            while (npend >= 8) {                                 // uniform
                cp_steps<MODEL>(&S.sp[CP_SP * (head >> 1) + 8 * js], &S.sf[CP_SF * (head >> 1) + 2 * js], 4, pi, mi,
                                A, phi, ax, ay, az);
                head = (head + 8) & 63;
                npend -= 8;
            }
            __syncwarp();
        }
    }
    if (npend > 0) {
        if ((npend & 1) && lane < 4) {
            // pad cluster: charge zero, 2a beyond the box in x (out of range of every
            // lane, finite distances: exact zero terms)
            const int q = (head + npend) & 63;
            float *e = &S.sp[CP_SP * (q >> 1) + 8 * lane + 1];
            e[0] = lo[0] - 2.f * A.a; e[2] = 0.5f * (lo[1] + hi[1]); e[4] = 0.5f * (lo[2] + hi[2]); e[6] = 0.f;
            S.sf[CP_SF * (q >> 1) + 2 * lane + 1] = -2;
        }
        __syncwarp();
        cp_steps<MODEL>(&S.sp[CP_SP * (head >> 1) + 8 * js], &S.sf[CP_SF * (head >> 1) + 2 * js], (npend + 1) >> 1, pi, mi, A, phi, ax, ay,
                        az);
    }
    // the four j slots of each i atom: lanes i, i + 8, i + 16, i + 24
#pragma unroll
    for (int o = 8; o < 32; o <<= 1) {
        phi += __shfl_xor_sync(0xffffffffu, phi, o);
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    if (valid && js == 0) {
        const int atom = A.perm[slot];
        A.sr[atom] = vec4<float>{-pi.w * ax, -pi.w * ay, -pi.w * az, phi};
        if (MODEL && !(A.aflag[slot] & 1)) A.lj[atom] = vec4<float>{0.f, 0.f, 0.f, 0.f};
    }
}

int launch_cluster_build(const ClusterArgs &a, bool model, cudaStream_t st)
{
    if (a.max_cols <= 0) return MSM_OK;
    const dim3 grid((a.max_cols + 3) / 4, a.bt.B);
    k_cp_count<<<grid, 128, 0, st>>>(a.bt, a.start, a.zc, a.col_n, a.status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    {
        const int rc = launch_scan(a.n_cols, a.col_n, a.col_cl, a.bsum, a.status, st);
        if (rc != MSM_OK) return rc;
    }
    if (model) k_cp_fill<true><<<grid, 128, 0, st>>>(a);
    else k_cp_fill<false><<<grid, 128, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

int launch_cluster_short(const ClusterArgs &a, bool model, cudaStream_t st)
{
    if (a.max_icl <= 0) return MSM_OK;
    const dim3 grid(a.max_icl, a.bt.B);
    if (model) k_cp_short<true><<<grid, 32, 0, st>>>(a);
    else k_cp_short<false><<<grid, 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

}  // namespace msm
