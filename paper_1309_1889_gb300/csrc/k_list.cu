// k_list.cu -- Verlet lists for the short-range part of the MSM (Sec. 3, step
// 1: u_i^short = sum_{r_ij < a} q_j g*(r_ij)) across velocity-Verlet steps.
//
// The same sum as k_short, organised so that a lane only visits the j atoms
// that were within a + skin of its i atom when the list was built.  A list
// stays exact while no atom has moved more than skin/2 since the build: every
// pair inside a is then in it, and the r < a test is still applied per pair.
//
// Reference frame: at a build the current cell sort (perm, cell_start) is
// frozen as the list's reference order, and every step gathers that step's
// positions into it (vl_pos).  The build runs the cell search of k_short -- one
// warp per brick, the brick's candidate rows (within a + skin of its atoms'
// bounding box) compacted into a row table, the row stream staged 32 atoms at
// a time and broadcast -- but instead of summing it appends every j within
// a + skin (other molecules only) to the lane's list.  An entry is 16 bits:
// the row's index in the brick's row table (9 bits) and the atom's offset in
// the row (7 bits).  Entries go four to a 64-bit word, and word q of slot s is
// stored at [q * n + s], so that the lanes of a warp read their words side by
// side.  O-O pairs of the water completion also go to a second, shorter list
// for the LJ term.
//
// The force kernel is one warp per brick again: the brick's row table in
// shared memory, each lane walking its own list and reading its j positions
// through the L1 cache.  Each lane adds its pairs in list order, i.e. in
// ascending reference slot order.
//
// Device flags (ctl): [0] max displacement^2 bits this step, [1] overflow
// (sticky until the host grows the buffers), [2] list invalid, [3] rebuild
// this step, [4] largest entries per atom seen, [5] largest O-O entries seen,
// [6] largest row count seen, [7] builds.  No kernel waits on another: each
// reads the flags written by earlier launches in the stream and returns early
// when it has nothing to do, so a step never needs a host synchronisation.
#include <stdint.h>

#include <algorithm>

#include "kernels.cuh"

namespace msm {

constexpr int VL_WARPS = 4;         // bricks per CTA

__device__ __forceinline__ bool vl_rebuild(const int *ctl) { return ctl[3] != 0; }
__device__ __forceinline__ bool vl_usable(const int *ctl) { return ctl[1] == 0 && ctl[2] == 0; }

template <typename T> __device__ __forceinline__ T vl_rsqrt(T x);
template <> __device__ __forceinline__ float vl_rsqrt<float>(float x) { return rsqrt_ftz(x); }
template <> __device__ __forceinline__ double vl_rsqrt<double>(double x) { return rsqrt(x); }
// added to r^2 through the FMA chain: keeps rsqrt finite for masked entries
template <typename T> __device__ __forceinline__ T vl_eps();
template <> __device__ __forceinline__ float vl_eps<float>() { return 1e-12f; }
template <> __device__ __forceinline__ double vl_eps<double>() { return 1e-30; }

// ------------------------------------------------------------ displacement

template <typename T>
__global__ void k_list_disp(ListArgs<T> A)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d2 = 0.f;
    if (i < A.n && A.ctl[2] == 0) {
        const double dx = A.x[3 * i] - A.vl_xref[3 * i], dy = A.x[3 * i + 1] - A.vl_xref[3 * i + 1],
                     dz = A.x[3 * i + 2] - A.vl_xref[3 * i + 2];
        d2 = (float)(dx * dx + dy * dy + dz * dz);
    }
    __shared__ float sm[8];
#pragma unroll
    for (int o = 16; o; o >>= 1) d2 = fmaxf(d2, __shfl_xor_sync(0xffffffffu, d2, o));
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = d2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) m = fmaxf(m, sm[w]);
        if (m > 0.f) atomicMax(&A.ctl[0], __float_as_int(m));   // m >= 0: int order = float order
    }
}

// Freeze the reference order when the list is invalid or an atom moved more than skin/2.
template <typename T>
__global__ void k_list_snapshot(ListArgs<T> A)
{
    if (failed(A.status)) return;
    const bool rebuild = A.ctl[1] == 0 && (A.ctl[2] != 0 || __int_as_float(A.ctl[0]) > (float)A.skin_half2);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        A.ctl[3] = rebuild ? 1 : 0;
        if (rebuild) A.ctl[7] += 1;                 // builds since the host last read the flags
    }
    if (!rebuild) return;
    if (i < A.n) {
        A.vl_perm[i] = A.perm[i];
        A.vl_xref[3 * i] = A.x[3 * i]; A.vl_xref[3 * i + 1] = A.x[3 * i + 1]; A.vl_xref[3 * i + 2] = A.x[3 * i + 2];
    }
    for (int c = i; c <= A.g.ncells; c += gridDim.x * blockDim.x) A.vl_start[c] = A.start[c];
}

// ------------------------------------------------------------------ build

// i atoms of brick (bx, by, bz) in the order of the cell-search kernel; returns
// the want-th atom's slot (or -1) and, in *count, the brick's atom count
__device__ __forceinline__ int brick_slot(const int *__restrict__ start, const CellGeom &g, const int bd[3], int bx,
                                          int by, int bz, int want, int *count)
{
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int cx0 = bx * bd[0], cx1 = min(cx0 + bd[0], nx);
    const int cy0 = by * bd[1], cy1 = min(cy0 + bd[1], ny);
    const int cz0 = bz * bd[2], cz1 = min(cz0 + bd[2], nz);
    int slot = -1, acc = 0;
    for (int cz = cz0; cz < cz1; cz++)
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            const int s0 = start[rb + cx0], c = start[rb + cx1] - s0;
            if (slot < 0 && want >= acc && want < acc + c) slot = s0 + (want - acc);
            acc += c;
        }
    *count = acc;
    return slot;
}

template <typename T>
__device__ __forceinline__ T warp_minv(T v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

struct VLBuildSmem {
    int rs0[VL_WARPS][VL_ROWS];     // first slot of each candidate row
    int rend[VL_WARPS][VL_ROWS];    // running end of each row in the row stream
};

template <typename T>
__global__ void __launch_bounds__(VL_WARPS * 32) k_list_build(ListArgs<T> A)
{
    __shared__ VLBuildSmem S;
    __shared__ vec4<T> sj[VL_WARPS][32];
    __shared__ int sf[VL_WARPS][32], ss[VL_WARPS][32], sc[VL_WARPS][32];
    if (!vl_rebuild(A.ctl) || failed(A.status)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int brick = blockIdx.x * VL_WARPS + wid;
    if (brick >= A.nbricks) return;
    const unsigned lt = (1u << lane) - 1u;
    const CellGeom &G = A.g;
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int bx = brick % A.nb[0], by = (brick / A.nb[0]) % A.nb[1], bz = brick / (A.nb[0] * A.nb[1]);
    const T h = (T)G.h, inv_h = T(1) / h;

    // bounding box of all the brick's atoms
    int n_i = 0;
    brick_slot(A.start, G, A.bd, bx, by, bz, 0, &n_i);
    if (n_i == 0) { if (lane == 0) A.rtn[brick] = 0; return; }
    T lo[3] = {(T)1e30, (T)1e30, (T)1e30}, nhi[3] = {(T)1e30, (T)1e30, (T)1e30};   // nhi: -max
    for (int base = 0; base < n_i; base += 32) {
        int c;
        const int sl = brick_slot(A.start, G, A.bd, bx, by, bz, base + lane, &c);
        const bool ok = sl >= 0;
        const vec4<T> p = ok ? A.apos[sl] : vec4<T>{(T)0, (T)0, (T)0, (T)0};
        lo[0] = min(lo[0], warp_minv(ok ? p.x : (T)1e30));
        lo[1] = min(lo[1], warp_minv(ok ? p.y : (T)1e30));
        lo[2] = min(lo[2], warp_minv(ok ? p.z : (T)1e30));
        nhi[0] = min(nhi[0], warp_minv(ok ? -p.x : (T)1e30));
        nhi[1] = min(nhi[1], warp_minv(ok ? -p.y : (T)1e30));
        nhi[2] = min(nhi[2], warp_minv(ok ? -p.z : (T)1e30));
    }
    const T hi[3] = {-nhi[0], -nhi[1], -nhi[2]};

    // candidate rows within a + skin of the box, compacted into the row table
    const T rs = A.rl_sel, rs2 = rs * rs;
    const int zlo = max(0, (int)floor((lo[2] - rs) * inv_h)), zhi = min(nz - 1, (int)floor((hi[2] + rs) * inv_h));
    const int ylo = max(0, (int)floor((lo[1] - rs) * inv_h)), yhi = min(ny - 1, (int)floor((hi[1] + rs) * inv_h));
    const int nyr = yhi - ylo + 1, nr_all = max(0, zhi - zlo + 1) * max(0, nyr);
    int nrows = 0, total = 0;
    bool bad = false;
    for (int r0 = 0; r0 < nr_all; r0 += 32) {
        const int r = r0 + lane;
        int s0 = 0, len = 0;
        if (r < nr_all) {
            const int cz = zlo + r / nyr, cy = ylo + r % nyr;
            const T dz = max(T(0), max(T(cz) * h - hi[2], lo[2] - T(cz + 1) * h));
            const T dy = max(T(0), max(T(cy) * h - hi[1], lo[1] - T(cy + 1) * h));
            const T d2 = dy * dy + dz * dz;
            if (d2 < rs2) {
                const T rx = sqrt(rs2 - d2);
                const int xlo = max(0, (int)floor((lo[0] - rx) * inv_h));
                const int xhi = min(nx - 1, (int)floor((hi[0] + rx) * inv_h));
                if (xlo <= xhi) {
                    const int rb = (cz * ny + cy) * nx;
                    s0 = A.start[rb + xlo];
                    len = A.start[rb + xhi + 1] - s0;
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, len > 0);
        bad = bad || __any_sync(0xffffffffu, len >= VL_OFFS);
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const int pos = nrows + __popc(m & lt);
        if (len > 0 && pos < VL_ROWS) {
            S.rs0[wid][pos] = s0;
            S.rend[wid][pos] = total + incl;
            A.rtab[(size_t)brick * VL_ROWS + pos] = s0;
        }
        nrows += __popc(m);
        total += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        atomicMax(&A.ctl[6], nrows);
        A.rtn[brick] = min(nrows, VL_ROWS);
    }
    if (nrows > VL_ROWS || bad) {                 // the entry code cannot address this brick
        if (lane == 0) A.ctl[1] = 1;
        return;
    }
    __syncwarp();

    const T rl2 = A.rl2;
    const size_t n = (size_t)A.n;
    for (int base = 0; base < n_i; base += 32) {
        int dummy;
        const int sI = brick_slot(A.start, G, A.bd, bx, by, bz, base + lane, &dummy);
        const bool valid = sI >= 0;
        const vec4<T> pi = valid ? A.apos[sI] : vec4<T>{(T)1e30, (T)1e30, (T)1e30, (T)0};
        const int fi = valid ? A.aflag[sI] : -2;
        unsigned long long qc = 0ull, ql = 0ull;
        int c = 0, cl = 0;
        bool over = false;
        for (int cb = 0; cb < total; cb += 32) {
            const int cnt = min(32, total - cb);
            if (lane < cnt) {
                const int want = cb + lane;
                int lo_r = 0, hi_r = nrows - 1;
                while (lo_r < hi_r) {
                    const int mid = (lo_r + hi_r) >> 1;
                    if (S.rend[wid][mid] > want) hi_r = mid; else lo_r = mid + 1;
                }
                const int off = want - (lo_r ? S.rend[wid][lo_r - 1] : 0);
                const int js = S.rs0[wid][lo_r] + off;
                sj[wid][lane] = A.apos[js];
                sf[wid][lane] = A.aflag[js];
                ss[wid][lane] = js;
                sc[wid][lane] = (lo_r << 7) | off;
            }
            __syncwarp();
            for (int k = 0; k < cnt; k++) {
                const vec4<T> pj = sj[wid][k];
                const int fj = sf[wid][k];
                const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                bool take = valid && r2 < rl2;
                if (A.model) take = take && ((unsigned)(fi ^ fj) >= 2u);     // other molecules (and j != i)
                else take = take && ss[wid][k] != sI;
                if (take) {
                    const unsigned long long code = (unsigned long long)sc[wid][k];
                    if (c < A.cap) {
                        qc |= code << (16 * (c & 3));
                        if ((c & 3) == 3) { A.nbr[(size_t)(c >> 2) * n + sI] = qc; qc = 0ull; }
                    } else over = true;
                    c++;
                    if (A.model && (fi & fj & 1)) {
                        if (cl < A.cap_lj) {
                            ql |= code << (16 * (cl & 3));
                            if ((cl & 3) == 3) { A.nbr_lj[(size_t)(cl >> 2) * n + sI] = ql; ql = 0ull; }
                        } else over = true;
                        cl++;
                    }
                }
            }
            __syncwarp();
        }
        if (valid) {
            if ((c & 3) && c < A.cap) A.nbr[(size_t)(c >> 2) * n + sI] = qc;
            if ((cl & 3) && cl < A.cap_lj) A.nbr_lj[(size_t)(cl >> 2) * n + sI] = ql;
            A.cnt[sI] = c;
            A.cntlj[sI] = cl;
        }
        int mc = valid ? c : 0, ml = valid ? cl : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            mc = max(mc, __shfl_xor_sync(0xffffffffu, mc, o));
            ml = max(ml, __shfl_xor_sync(0xffffffffu, ml, o));
        }
        const bool any_over = __any_sync(0xffffffffu, over);
        if (lane == 0) {
            atomicMax(&A.ctl[4], mc);
            atomicMax(&A.ctl[5], ml);
            if (any_over) A.ctl[1] = 1;
        }
    }
}

// Reference-ordered positions of the current step (and the end of a build).
template <typename T>
__global__ void k_list_gather(ListArgs<T> A)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (failed(A.status) || A.ctl[1] != 0) return;
    if (s == 0 && A.ctl[3] != 0) A.ctl[2] = 0;                  // a build completed without overflow: valid
    if (A.ctl[2] != 0 && A.ctl[3] == 0) return;
    if (s >= A.n) return;
    const int i = A.vl_perm[s];
    A.vl_pos[s] = vec4<T>{(T)(A.x[3 * i] - A.g.origin[0]), (T)(A.x[3 * i + 1] - A.g.origin[1]),
                          (T)(A.x[3 * i + 2] - A.g.origin[2]), (T)A.q[i]};
}

// ------------------------------------------------------------------ forces

template <typename T, bool MODEL>
__global__ void __launch_bounds__(VL_WARPS * 32) k_short_list(ListArgs<T> A)
{
    __shared__ int rt[VL_WARPS][VL_ROWS];
    if (!vl_usable(A.ctl) || failed(A.status)) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int brick = blockIdx.x * VL_WARPS + wid;
    if (brick >= A.nbricks) return;
    const int nrows = A.rtn[brick];
    if (nrows == 0) return;
    for (int r = lane; r < nrows; r += 32) rt[wid][r] = A.rtab[(size_t)brick * VL_ROWS + r];
    __syncwarp();
    const int bx = brick % A.nb[0], by = (brick / A.nb[0]) % A.nb[1], bz = brick / (A.nb[0] * A.nb[1]);
    int n_i = 0;
    brick_slot(A.vl_start, A.g, A.bd, bx, by, bz, 0, &n_i);
    const T a2 = A.a2;
    const size_t n = (size_t)A.n;
    const vec4<T> *__restrict__ P = A.vl_pos;
    for (int base = 0; base < n_i; base += 32) {
        int dummy;
        const int sI = brick_slot(A.vl_start, A.g, A.bd, bx, by, bz, base + lane, &dummy);
        const bool valid = sI >= 0;
        const int self = valid ? sI : 0;
        const vec4<T> pi = valid ? P[sI] : vec4<T>{(T)1e30, (T)1e30, (T)1e30, (T)0};
        const int cnt = valid ? A.cnt[sI] : 0;
        int maxc = cnt;
#pragma unroll
        for (int o = 16; o; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
        T phi = 0, ax = 0, ay = 0, az = 0;
        unsigned long long nxt = cnt > 0 ? A.nbr[self] : 0ull;
        for (int k4 = 0; k4 < maxc; k4 += 4) {
            const unsigned long long w = nxt;
            if (k4 + 4 < cnt) nxt = A.nbr[(size_t)((k4 >> 2) + 1) * n + sI];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int code = (int)((w >> (16 * e)) & 0xffffull);
                const bool act = k4 + e < cnt;
                const vec4<T> pj = P[act ? rt[wid][code >> 7] + (code & 127) : self];
                const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const T r2s = fma(dx, dx, fma(dy, dy, fma(dz, dz, vl_eps<T>())));
                const T qj = (act && r2s < a2) ? pj.w : T(0);
                const T ri = vl_rsqrt<T>(r2s);
                const T ri2 = ri * ri;
                const T poly = fma(fma(A.c2, r2s, A.c1), r2s, A.c0);
                phi = fma(qj, ri - poly, phi);
                const T fs = fma(ri2, ri, fma(A.d1, r2s, A.d0));
                const T sc = qj * fs;
                ax = fma(sc, dx, ax); ay = fma(sc, dy, ay); az = fma(sc, dz, az);
            }
        }
        T lx = 0, ly = 0, lz = 0, le = 0;
        if (MODEL) {
            const int cl = valid ? A.cntlj[sI] : 0;
            int maxl = cl;
#pragma unroll
            for (int o = 16; o; o >>= 1) maxl = max(maxl, __shfl_xor_sync(0xffffffffu, maxl, o));
            unsigned long long nl = cl > 0 ? A.nbr_lj[self] : 0ull;
            for (int k4 = 0; k4 < maxl; k4 += 4) {
                const unsigned long long w = nl;
                if (k4 + 4 < cl) nl = A.nbr_lj[(size_t)((k4 >> 2) + 1) * n + sI];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int code = (int)((w >> (16 * e)) & 0xffffull);
                    const bool act = k4 + e < cl;
                    const vec4<T> pj = P[act ? rt[wid][code >> 7] + (code & 127) : self];
                    const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const T r2s = fma(dx, dx, fma(dy, dy, fma(dz, dz, vl_eps<T>())));
                    const bool on = act && r2s < a2;
                    const T ri = vl_rsqrt<T>(r2s);
                    const T ir2 = on ? ri * ri : T(0);
                    const T sr2 = A.lj_s2 * ir2;
                    const T sr6 = sr2 * sr2 * sr2;
                    const T m = on ? T(1) : T(0);
                    le = fma(m, fma(A.lj_4eps, sr6 * sr6 - sr6, -A.lj_shift), le);
                    const T fl = A.lj_24eps * fma(T(2) * sr6, sr6, -sr6) * ir2;
                    lx = fma(-fl, dx, lx); ly = fma(-fl, dy, ly); lz = fma(-fl, dz, lz);
                }
            }
        }
        if (valid) {
            const int i = A.vl_perm[sI];
            A.sr[i] = vec4<T>{-pi.w * ax, -pi.w * ay, -pi.w * az, phi};
            if (MODEL) A.lj[i] = vec4<T>{lx, ly, lz, le};
        }
    }
}

// ---------------------------------------------------------------- launches

template <typename T>
int launch_list_maintain(const ListArgs<T> &a, cudaStream_t st)
{
    const int n = a.n;
    CUDA_TRY(cudaMemsetAsync(a.ctl, 0, sizeof(int), st));                // ctl[0]: this step's max displacement
    if (n > 0) k_list_disp<T><<<(n + 255) / 256, 256, 0, st>>>(a);
    const int m = std::max(n, a.g.ncells + 1);
    k_list_snapshot<T><<<(m + 255) / 256, 256, 0, st>>>(a);
    if (a.nbricks > 0) k_list_build<T><<<(a.nbricks + VL_WARPS - 1) / VL_WARPS, VL_WARPS * 32, 0, st>>>(a);
    k_list_gather<T><<<(n + 255) / 256 + 1, 256, 0, st>>>(a);
    count_launch((n > 0 ? 3 : 2) + (a.nbricks > 0 ? 1 : 0));
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_list_force(const ListArgs<T> &a, cudaStream_t st)
{
    const int grid = (a.nbricks + VL_WARPS - 1) / VL_WARPS;
    if (grid <= 0) return MSM_OK;
    if (a.model) k_short_list<T, true><<<grid, VL_WARPS * 32, 0, st>>>(a);
    else k_short_list<T, false><<<grid, VL_WARPS * 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_list_maintain<float>(const ListArgs<float> &, cudaStream_t);
template int launch_list_maintain<double>(const ListArgs<double> &, cudaStream_t);
template int launch_list_force<float>(const ListArgs<float> &, cudaStream_t);
template int launch_list_force<double>(const ListArgs<double> &, cudaStream_t);

}  // namespace msm
