// k_list.cu -- Verlet lists for the short-range part of the MSM (Sec. 3, step
// 1: u_i^short = sum_{r_ij < a} q_j g*(r_ij)) across velocity-Verlet steps.
//
// The same sum as k_short, organised so that a lane only visits the j atoms
// that were within a + skin of its i atom when the list was built.  A list
// stays exact while no atom has moved more than skin/2 since the build: every
// pair inside a is then in it, and the r < a test is still applied per pair.
//
// Reference frame: at a build, the current cell sort (perm, cell_start) is
// frozen as the list's reference order.  A group = 2 x 2 bricks in (y, z)
// (one brick per warp, the bricks of the cell-search kernel) shares one
// neighbourhood J: the cell rows within a + skin of the group's atom bounding
// box, each one contiguous range of reference slots.  List entries are uint16
// indices into J, which is staged in shared memory every step; Coulomb
// entries run forward from slot * cap, O-O LJ entries backward from
// slot * cap + cap - 1.  Intramolecular pairs of the water completion are
// left out at build time.
//
// Device flags (ctl): [0] max displacement^2 bits this step, [1] overflow
// (sticky until the host grows the buffers), [2] list invalid, [3] rebuild
// this step, [4] largest entries per atom seen, [5] largest neighbourhood
// seen, [6] largest row count seen.  No kernel waits on another: each one
// reads the flags written by earlier launches in the stream and returns early
// when it has nothing to do, so a step never needs a host synchronisation.
#include <stdint.h>

#include <algorithm>

#include "kernels.cuh"

namespace msm {

constexpr int VL_WARPS = 4;         // bricks (by + wy, bz + wz), wy, wz in {0, 1}

__device__ __forceinline__ bool vl_rebuild(const int *ctl) { return ctl[3] != 0; }
__device__ __forceinline__ bool vl_usable(const int *ctl) { return ctl[1] == 0 && ctl[2] == 0; }

template <typename T> __device__ __forceinline__ T vl_rsqrt(T x);
template <> __device__ __forceinline__ float vl_rsqrt<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double vl_rsqrt<double>(double x) { return rsqrt(x); }

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

struct VLRow { int y, z, s0, len, base, xlo, xhi, pad; };

template <typename T>
__device__ __forceinline__ void warp_bbox(bool valid, const vec4<T> &p, T lo[3], T hi[3])
{
    const T inf = (T)1e30;
    T v[6] = {valid ? p.x : inf, valid ? p.y : inf, valid ? p.z : inf,
              valid ? -p.x : inf, valid ? -p.y : inf, valid ? -p.z : inf};
#pragma unroll
    for (int k = 0; k < 6; k++)
#pragma unroll
        for (int o = 16; o; o >>= 1) v[k] = min(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
    lo[0] = v[0]; lo[1] = v[1]; lo[2] = v[2]; hi[0] = -v[3]; hi[1] = -v[4]; hi[2] = -v[5];
}

// i atoms of brick (bx, by, bz) in the order of the cell-search kernel; returns their count and,
// for lane-th atom of chunk base, its slot (or -1)
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
__global__ void __launch_bounds__(VL_WARPS * 32) k_list_build(ListArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!vl_rebuild(A.ctl) || failed(A.status)) return;
    vec4<T> *sJ = reinterpret_cast<vec4<T> *>(smem_raw);                  // jcap
    int *sF = reinterpret_cast<int *>(sJ + A.jcap);                        // jcap flags
    VLRow *sR = reinterpret_cast<VLRow *>(sF + A.jcap);                    // max_rows
    uint16_t *sB = reinterpret_cast<uint16_t *>(sR + A.max_rows);          // VL_WARPS x 32 x 16 write buffers
    __shared__ T s_bb[VL_WARPS][6];
    __shared__ int s_cnt[VL_WARPS];
    __shared__ int s_nrows, s_J, s_bad;

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = blockIdx.x;
    const int gx = g % A.ng[0], gyb = (g / A.ng[0]) % A.ng[1], gzb = g / (A.ng[0] * A.ng[1]);
    const int bx = gx, by = 2 * gyb + (wid & 1), bz = 2 * gzb + (wid >> 1);
    const bool brick_ok = by < A.nb[1] && bz < A.nb[2];
    const CellGeom &G = A.g;
    const T h = (T)G.h, inv_h = T(1) / h;

    // bounding box of each brick's atoms (all chunks)
    int n_i = 0;
    if (brick_ok) brick_slot(A.start, G, A.bd, bx, by, bz, 0, &n_i);
    T blo[3] = {(T)1e30, (T)1e30, (T)1e30}, bhi[3] = {(T)-1e30, (T)-1e30, (T)-1e30};
    for (int base = 0; base < n_i; base += 32) {
        int c;
        const int sl = brick_slot(A.start, G, A.bd, bx, by, bz, base + lane, &c);
        const vec4<T> p = sl >= 0 ? A.apos[sl] : vec4<T>{0, 0, 0, 0};
        T lo[3], hi[3];
        warp_bbox(sl >= 0, p, lo, hi);
#pragma unroll
        for (int d = 0; d < 3; d++) { blo[d] = min(blo[d], lo[d]); bhi[d] = max(bhi[d], hi[d]); }
    }
    if (lane == 0) {
        s_cnt[wid] = n_i;
#pragma unroll
        for (int d = 0; d < 3; d++) { s_bb[wid][d] = blo[d]; s_bb[wid][3 + d] = bhi[d]; }
    }
    __syncthreads();

    // union rows (warp 0): cell rows within a + skin of the union box
    if (wid == 0) {
        T ulo[3] = {(T)1e30, (T)1e30, (T)1e30}, uhi[3] = {(T)-1e30, (T)-1e30, (T)-1e30};
        int tot = 0;
        for (int w = 0; w < VL_WARPS; w++)
            if (s_cnt[w] > 0) {
                tot += s_cnt[w];
#pragma unroll
                for (int d = 0; d < 3; d++) { ulo[d] = min(ulo[d], s_bb[w][d]); uhi[d] = max(uhi[d], s_bb[w][3 + d]); }
            }
        int nrows = 0, J = 0, bad = 0;
        if (tot > 0) {
            const T rs = A.rl_sel, rs2 = rs * rs;
            const int zlo = max(0, (int)floor((ulo[2] - rs) * inv_h)), zhi = min(G.nc[2] - 1, (int)floor((uhi[2] + rs) * inv_h));
            const int ylo = max(0, (int)floor((ulo[1] - rs) * inv_h)), yhi = min(G.nc[1] - 1, (int)floor((uhi[1] + rs) * inv_h));
            const int ny = yhi - ylo + 1, cnt_rows = (zhi - zlo + 1) * ny;
            for (int r0 = 0; r0 < cnt_rows; r0 += 32) {
                const int r = r0 + lane;
                int keep = 0, s0 = 0, len = 0, xlo = 0, xhi = -1, cy = 0, cz = 0;
                if (r < cnt_rows) {
                    cz = zlo + r / ny; cy = ylo + r % ny;
                    const T dz = max(T(0), max(T(cz) * h - uhi[2], ulo[2] - T(cz + 1) * h));
                    const T dy = max(T(0), max(T(cy) * h - uhi[1], ulo[1] - T(cy + 1) * h));
                    const T d2 = dy * dy + dz * dz;
                    if (d2 < rs2) {
                        const T rx = sqrt(rs2 - d2);
                        xlo = max(0, (int)floor((ulo[0] - rx) * inv_h));
                        xhi = min(G.nc[0] - 1, (int)floor((uhi[0] + rx) * inv_h));
                        if (xlo <= xhi) {
                            const int rb = (cz * G.nc[1] + cy) * G.nc[0];
                            s0 = A.start[rb + xlo];
                            len = A.start[rb + xhi + 1] - s0;
                            keep = 1;
                        }
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, keep);
                int incl = len;                                        // inclusive scan of len over kept lanes
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) { const int y = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += y; }
                const int pos = nrows + __popc(m & ((1u << lane) - 1));
                if (keep) {
                    if (pos < A.max_rows) {
                        VLRow row;
                        row.y = cy; row.z = cz; row.s0 = s0; row.len = len; row.base = J + incl - len;
                        row.xlo = xlo; row.xhi = xhi; row.pad = 0;
                        sR[pos] = row;
                        A.grp_rows[(size_t)g * A.max_rows + pos] = make_int2(s0, len);
                    }
                }
                nrows += __popc(m);
                J += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (nrows > A.max_rows || J > A.jcap) bad = 1;
        }
        if (lane == 0) {
            s_nrows = nrows; s_J = J; s_bad = bad;
            A.grp_nrows[g] = bad ? 0 : nrows;
            A.grp_j[g] = bad ? 0 : J;
            if (bad) { A.ctl[1] = 1; atomicMax(&A.ctl[5], J); atomicMax(&A.ctl[6], nrows); }
        }
    }
    __syncthreads();
    if (s_bad || s_J == 0) return;
    const int nrows = s_nrows;

    // stage the neighbourhood: positions and (molecule, LJ) flags
    for (int r = wid; r < nrows; r += VL_WARPS) {
        const VLRow row = sR[r];
        for (int k = lane; k < row.len; k += 32) {
            sJ[row.base + k] = A.apos[row.s0 + k];
            sF[row.base + k] = A.aflag[row.s0 + k];
        }
    }
    __syncthreads();
    if (!brick_ok || n_i == 0) return;

    const T rl2 = A.rl2, rs = A.rl_sel, rs2 = rs * rs;
    uint16_t *bufC = sB + (wid * 2 + 0) * 32 * 8 + lane * 8;   // 8-entry write buffers per lane
    uint16_t *bufL = sB + (wid * 2 + 1) * 32 * 8 + lane * 8;
    for (int base = 0; base < n_i; base += 32) {
        int dummy;
        const int sI = brick_slot(A.start, G, A.bd, bx, by, bz, base + lane, &dummy);
        const bool valid = sI >= 0;
        const vec4<T> pi = valid ? A.apos[sI] : vec4<T>{(T)1e30, (T)1e30, (T)1e30, 0};
        const int fi = valid ? A.aflag[sI] : -2;
        T lo[3], hi[3];
        warp_bbox(valid, pi, lo, hi);
        uint16_t *row_out = A.nbr + (size_t)(valid ? sI : 0) * A.cap;
        int c = 0, cl = 0;
        bool over = false;
        for (int r = 0; r < nrows; r++) {
            const VLRow row = sR[r];
            // trim the union row to this chunk's box
            const T dz = max(T(0), max(T(row.z) * h - hi[2], lo[2] - T(row.z + 1) * h));
            const T dy = max(T(0), max(T(row.y) * h - hi[1], lo[1] - T(row.y + 1) * h));
            const T d2 = dy * dy + dz * dz;
            if (d2 >= rs2) continue;
            const T rx = sqrt(rs2 - d2);
            const int xlo = max(row.xlo, (int)floor((lo[0] - rx) * inv_h));
            const int xhi = min(row.xhi, (int)floor((hi[0] + rx) * inv_h));
            if (xlo > xhi) continue;
            const int rb = (row.z * G.nc[1] + row.y) * G.nc[0];
            const int j0 = row.base + (A.start[rb + xlo] - row.s0), j1 = row.base + (A.start[rb + xhi + 1] - row.s0);
            for (int j = j0; j < j1; j++) {
                const vec4<T> pj = sJ[j];
                const int fj = sF[j];
                const T ddx = pj.x - pi.x, ddy = pj.y - pi.y, ddz = pj.z - pi.z;
                const T r2 = ddx * ddx + ddy * ddy + ddz * ddz;
                const bool take = valid && r2 < rl2 && r2 > T(0) && (!A.model || ((fi ^ fj) >> 1) != 0);
                if (take && !over) {
                    if (c + cl + 16 > A.cap) {
                        over = true;
                    } else {
                        bufC[c & 7] = (uint16_t)j;
                        if ((c & 7) == 7) *reinterpret_cast<uint4 *>(row_out + (c & ~7)) = *reinterpret_cast<uint4 *>(bufC);
                        c++;
                        if (A.model && (fi & fj & 1)) {
                            bufL[cl & 7] = (uint16_t)j;
                            if ((cl & 7) == 7) *reinterpret_cast<uint4 *>(row_out + A.cap - 8 - (cl & ~7)) = *reinterpret_cast<uint4 *>(bufL);
                            cl++;
                        }
                    }
                }
            }
        }
        // flush partial buffers (the unused tail entries are never read: counts bound every read)
        if (valid && !over) {
            if (c & 7) *reinterpret_cast<uint4 *>(row_out + (c & ~7)) = *reinterpret_cast<uint4 *>(bufC);
            if (cl & 7) *reinterpret_cast<uint4 *>(row_out + A.cap - 8 - (cl & ~7)) = *reinterpret_cast<uint4 *>(bufL);
            A.cnt[sI] = c;
            A.cntlj[sI] = cl;
        }
        int used = valid ? c + cl + (over ? 1 : 0) : 0;
#pragma unroll
        for (int o = 16; o; o >>= 1) used = max(used, __shfl_xor_sync(0xffffffffu, used, o));
        if (lane == 0 && used > 0) atomicMax(&A.ctl[4], used);
        if (over) A.ctl[1] = 1;
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
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (!vl_usable(A.ctl) || failed(A.status)) return;
    vec4<T> *sJ = reinterpret_cast<vec4<T> *>(smem_raw);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = blockIdx.x;
    const int J = A.grp_j[g];
    if (J == 0) return;
    const int nrows = A.grp_nrows[g];
    const int2 *rows = A.grp_rows + (size_t)g * A.max_rows;
    // stage the group's neighbourhood from this step's reference-ordered positions
    {
        // rows are contiguous in the local index space in row order: recompute bases with a warp scan
        int base = 0;
        for (int r0 = 0; r0 < nrows; r0 += 32) {
            const int r = r0 + lane;
            const int2 rw = r < nrows ? rows[r] : make_int2(0, 0);
            int incl = rw.y;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) { const int y = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += y; }
            const int b = base + incl - rw.y;
            // each warp copies a quarter of the rows of this round
            for (int k = 0; k < 32; k++) {
                const int rr = r0 + k;
                if (rr >= nrows) break;
                const int bb = __shfl_sync(0xffffffffu, b, k);
                const int s0 = __shfl_sync(0xffffffffu, rw.x, k), len = __shfl_sync(0xffffffffu, rw.y, k);
                if ((k & (VL_WARPS - 1)) != wid) continue;
                for (int t = lane; t < len; t += 32) sJ[bb + t] = A.vl_pos[s0 + t];
            }
            base += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
    __syncthreads();
    const int gx = g % A.ng[0], gyb = (g / A.ng[0]) % A.ng[1], gzb = g / (A.ng[0] * A.ng[1]);
    const int bx = gx, by = 2 * gyb + (wid & 1), bz = 2 * gzb + (wid >> 1);
    if (by >= A.nb[1] || bz >= A.nb[2]) return;
    int n_i = 0;
    brick_slot(A.vl_start, A.g, A.bd, bx, by, bz, 0, &n_i);
    const T a2 = A.a2;
    for (int base = 0; base < n_i; base += 32) {
        int dummy;
        const int sI = brick_slot(A.vl_start, A.g, A.bd, bx, by, bz, base + lane, &dummy);
        const bool valid = sI >= 0;
        const vec4<T> pi = valid ? A.vl_pos[sI] : vec4<T>{(T)1e30, (T)1e30, (T)1e30, 0};
        const int cnt = valid ? A.cnt[sI] : 0;
        int maxc = cnt;
#pragma unroll
        for (int o = 16; o; o >>= 1) maxc = max(maxc, __shfl_xor_sync(0xffffffffu, maxc, o));
        const uint16_t *lst = A.nbr + (size_t)(valid ? sI : 0) * A.cap;
        T phi = 0, ax = 0, ay = 0, az = 0;
        uint4 nxt = make_uint4(0, 0, 0, 0);
        if (0 < cnt) nxt = __ldcs(reinterpret_cast<const uint4 *>(lst));
        for (int k8 = 0; k8 < maxc; k8 += 8) {
            const uint4 v = nxt;
            if (k8 + 8 < cnt) nxt = __ldcs(reinterpret_cast<const uint4 *>(lst + k8 + 8));
            const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const int j = (w[e >> 1] >> ((e & 1) * 16)) & 0xffff;
                const bool act = k8 + e < cnt;
                const vec4<T> pj = sJ[act ? j : 0];
                const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                const bool in = act & (r2 < a2);
                const T r2s = in ? r2 : a2;
                const T qj = in ? pj.w : T(0);
                const T ri = vl_rsqrt<T>(r2s);
                const T ri2 = ri * ri;
                const T poly = fma(fma(A.c2, r2s, A.c1), r2s, A.c0);
                phi = fma(qj, ri - poly, phi);
                const T fs = fma(ri2, ri, fma(A.d1, r2s, A.d0));
                const T s = qj * fs;
                ax = fma(s, dx, ax); ay = fma(s, dy, ay); az = fma(s, dz, az);
            }
        }
        T lx = 0, ly = 0, lz = 0, le = 0;
        if (MODEL) {
            const int cl = valid ? A.cntlj[sI] : 0;
            int maxl = cl;
#pragma unroll
            for (int o = 16; o; o >>= 1) maxl = max(maxl, __shfl_xor_sync(0xffffffffu, maxl, o));
            uint4 nl = make_uint4(0, 0, 0, 0);
            if (0 < cl) nl = __ldcs(reinterpret_cast<const uint4 *>(lst + A.cap - 8));
            for (int k8 = 0; k8 < maxl; k8 += 8) {
                const uint4 v = nl;
                if (k8 + 8 < cl) nl = __ldcs(reinterpret_cast<const uint4 *>(lst + A.cap - 16 - k8));
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 8; e++) {
                    // LJ entry k sits at cap - 8 - 8 floor(k/8) + (k mod 8): position e of block k8
                    const int j = (w[e >> 1] >> ((e & 1) * 16)) & 0xffff;
                    const bool act = k8 + e < cl;
                    const vec4<T> pj = sJ[act ? j : 0];
                    const T dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const T r2 = fma(dx, dx, fma(dy, dy, dz * dz));
                    const bool in = act & (r2 < a2);
                    const T ir2 = T(1) / (in ? r2 : a2);
                    const T sr2 = A.lj_s2 * ir2;
                    const T sr6 = sr2 * sr2 * sr2;
                    const T m = in ? T(1) : T(0);
                    le = fma(m, fma(A.lj_4eps, sr6 * sr6 - sr6, -A.lj_shift), le);
                    const T fl = m * A.lj_24eps * fma(T(2) * sr6, sr6, -sr6) * ir2;
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

template <typename T> size_t list_build_smem(const ListArgs<T> &a)
{
    return (size_t)a.jcap * (sizeof(vec4<T>) + sizeof(int)) + (size_t)a.max_rows * sizeof(VLRow) +
           (size_t)VL_WARPS * 2 * 32 * 8 * sizeof(uint16_t);
}
template <typename T> size_t list_force_smem(const ListArgs<T> &a) { return (size_t)a.jcap * sizeof(vec4<T>); }

template <typename T>
int launch_list_maintain(const ListArgs<T> &a, cudaStream_t st)
{
    const int n = a.n;
    CUDA_TRY(cudaMemsetAsync(a.ctl, 0, sizeof(int), st));                // ctl[0]: this step's max displacement
    if (n > 0) k_list_disp<T><<<(n + 255) / 256, 256, 0, st>>>(a);
    const int m = std::max(n, a.g.ncells + 1);
    k_list_snapshot<T><<<(m + 255) / 256, 256, 0, st>>>(a);
    const size_t sb = list_build_smem(a);
    CUDA_TRY(cudaFuncSetAttribute(k_list_build<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb));
    k_list_build<T><<<a.ngroups, VL_WARPS * 32, sb, st>>>(a);
    k_list_gather<T><<<(n + 255) / 256 + 1, 256, 0, st>>>(a);
    count_launch(n > 0 ? 4 : 3);
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_list_force(const ListArgs<T> &a, cudaStream_t st)
{
    const size_t sf = list_force_smem(a);
    if (a.model) {
        CUDA_TRY(cudaFuncSetAttribute(k_short_list<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
        k_short_list<T, true><<<a.ngroups, VL_WARPS * 32, sf, st>>>(a);
    } else {
        CUDA_TRY(cudaFuncSetAttribute(k_short_list<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf));
        k_short_list<T, false><<<a.ngroups, VL_WARPS * 32, sf, st>>>(a);
    }
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_list_maintain<float>(const ListArgs<float> &, cudaStream_t);
template int launch_list_maintain<double>(const ListArgs<double> &, cudaStream_t);
template int launch_list_force<float>(const ListArgs<float> &, cudaStream_t);
template int launch_list_force<double>(const ListArgs<double> &, cudaStream_t);
template size_t list_build_smem<float>(const ListArgs<float> &);
template size_t list_build_smem<double>(const ListArgs<double> &);

}  // namespace msm
