// k_short.cu -- short-range part of the MSM (Sec. 3, step 1):
//   u_i^short = sum_{j != i, r_ij < a} q_j g*(r_ij),  g*(r) = 1/r - gamma(r/a)/a,
//   F_i^short = -q_i sum_j q_j g*'(r_ij) (r_i - r_j)/r_ij
//             =  q_i sum_j q_j [1/r^3 - 5/(2a^3) + 3r^2/(2a^5)] (r_i - r_j).
//
// Layout: atoms sorted by finest-grid cell (x fastest), so a run of cells
// along x is one contiguous slot range.  One warp owns one brick of
// bd[0] x bd[1] x bd[2] cells (about 24 atoms: one i-atom per lane).  The
// warp's j candidates are whole cell rows (fixed y, z) whose distance to the
// brick's atom bounding box is below a, each trimmed in x to the cells that
// can still lie within a: every row is one contiguous slot range, staged 32
// atoms at a time in shared memory and broadcast to all lanes.  Per candidate
// the lane evaluates one rsqrt and ~20 FP32 FMA-pipe instructions; pairs
// beyond a (or j = i) are masked by substitution, never by divergence.
// Each i sums its own j's in a fixed order: no atomics, bitwise reproducible.
#include "kernels.cuh"

namespace msm {

constexpr int SR_WARPS = 4;

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
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

// MODEL: rigid-water completion -- pairs inside one molecule are skipped (the
// exclusion kernel removes their smooth part), LJ between flagged sites.
// COUNT: diagnostics only -- count the pairs inside the cutoff instead of summing.
template <typename T, bool MODEL, bool COUNT>
__global__ void __launch_bounds__(SR_WARPS * 32) k_short(const ShortArgs<T> A)
{
    __shared__ vec4<T> sj[SR_WARPS][32];
    __shared__ int sf[SR_WARPS][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int brick = blockIdx.x * SR_WARPS + wid;
    if (brick >= A.nbricks || failed(A.status)) return;
    const int nx = A.g.nc[0], ny = A.g.nc[1], nz = A.g.nc[2];
    const int bx = brick % A.nb[0], by = (brick / A.nb[0]) % A.nb[1], bz = brick / (A.nb[0] * A.nb[1]);
    const int cx0 = bx * A.bd[0], cx1 = min(cx0 + A.bd[0], nx);
    const int cy0 = by * A.bd[1], cy1 = min(cy0 + A.bd[1], ny);
    const int cz0 = bz * A.bd[2], cz1 = min(cz0 + A.bd[2], nz);
    const int *__restrict__ start = A.start;

    int n_i = 0;
    for (int cz = cz0; cz < cz1; cz++)
        for (int cy = cy0; cy < cy1; cy++) {
            const int rb = (cz * ny + cy) * nx;
            n_i += start[rb + cx1] - start[rb + cx0];
        }
    const T h = (T)A.g.h, inv_h = T(1) / h;
    const T a_sel2 = A.a_sel * A.a_sel;

    for (int base = 0; base < n_i; base += 32) {
        // ---- this lane's i atom: the (base + lane)-th atom of the brick
        int slot = -1;
        {
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
        vec4<T> pi = valid ? A.apos[slot] : vec4<T>{big_t<T>(), big_t<T>(), big_t<T>(), T(0)};
        const int fi = (MODEL && valid) ? A.aflag[slot] : -2;

        // ---- bounding box of the valid i atoms
        T lo[3], hi[3];
        lo[0] = warp_min(valid ? pi.x : inf_t<T>()); hi[0] = warp_max(valid ? pi.x : -inf_t<T>());
        lo[1] = warp_min(valid ? pi.y : inf_t<T>()); hi[1] = warp_max(valid ? pi.y : -inf_t<T>());
        lo[2] = warp_min(valid ? pi.z : inf_t<T>()); hi[2] = warp_max(valid ? pi.z : -inf_t<T>());

        T phi = 0, ax = 0, ay = 0, az = 0;
        T lx = 0, ly = 0, lz = 0, le = 0;
        int npair = 0;

        const int zlo = max(0, (int)floor((lo[2] - A.a_sel) * inv_h));
        const int zhi = min(nz - 1, (int)floor((hi[2] + A.a_sel) * inv_h));
        const int ylo = max(0, (int)floor((lo[1] - A.a_sel) * inv_h));
        const int yhi = min(ny - 1, (int)floor((hi[1] + A.a_sel) * inv_h));
        for (int cz = zlo; cz <= zhi; cz++) {
            const T dz = max(T(0), max(T(cz) * h - hi[2], lo[2] - T(cz + 1) * h));
            for (int cy = ylo; cy <= yhi; cy++) {
                const T dy = max(T(0), max(T(cy) * h - hi[1], lo[1] - T(cy + 1) * h));
                const T dyz2 = dy * dy + dz * dz;
                if (dyz2 >= a_sel2) continue;
                const T rx = sqrt(a_sel2 - dyz2);
                const int xlo = max(0, (int)floor((lo[0] - rx) * inv_h));
                const int xhi = min(nx - 1, (int)floor((hi[0] + rx) * inv_h));
                if (xlo > xhi) continue;
                const int rb = (cz * ny + cy) * nx;
                const int s0 = start[rb + xlo], s1 = start[rb + xhi + 1];
                for (int jb = s0; jb < s1; jb += 32) {
                    const int cnt = min(32, s1 - jb);
                    if (lane < cnt) {
                        sj[wid][lane] = A.apos[jb + lane];
                        if (MODEL) sf[wid][lane] = A.aflag[jb + lane];
                    }
                    __syncwarp();
#pragma unroll 4
                    for (int k = 0; k < cnt; k++) {
                        const vec4<T> pj = sj[wid][k];
                        const T dx = pj.x - pi.x, dyy = pj.y - pi.y, dzz = pj.z - pi.z;
                        const T r2 = fma(dx, dx, fma(dyy, dyy, dzz * dzz));
                        bool in = (r2 < A.a2) & (r2 > T(0));
                        int fj = 0;
                        if (MODEL) { fj = sf[wid][k]; in = in & (((fi ^ fj) >> 1) != 0); }
                        if (COUNT) { npair += in ? 1 : 0; continue; }
                        const T r2s = in ? r2 : A.a2;
                        const T qj = in ? pj.w : T(0);
                        const T ri = rsqrt_t<T>(r2s);
                        const T ri2 = ri * ri;
                        const T poly = fma(fma(A.c2, r2s, A.c1), r2s, A.c0);
                        phi = fma(qj, ri - poly, phi);
                        const T fs = fma(ri2, ri, fma(A.d1, r2s, A.d0));
                        const T s = qj * fs;
                        ax = fma(s, dx, ax); ay = fma(s, dyy, ay); az = fma(s, dzz, az);
                        if (MODEL) {
                            if (fj & 1) {
                                const T m = ((fi & 1) && in) ? T(1) : T(0);
                                const T sr2 = A.lj_s2 * ri2;
                                const T sr6 = sr2 * sr2 * sr2;
                                le = fma(m, fma(A.lj_4eps, sr6 * sr6 - sr6, -A.lj_shift), le);
                                const T fl = m * A.lj_24eps * fma(T(2) * sr6, sr6, -sr6) * ri2;
                                lx = fma(-fl, dx, lx); ly = fma(-fl, dyy, ly); lz = fma(-fl, dzz, lz);
                            }
                        }
                    }
                    __syncwarp();
                }
            }
        }
        if (valid) {
            if (COUNT) { A.cnt[slot] = (double)npair; continue; }
            A.sr[slot] = vec4<T>{-pi.w * ax, -pi.w * ay, -pi.w * az, phi};
            if (MODEL) A.lj[slot] = vec4<T>{lx, ly, lz, le};
        }
    }
}

template <typename T>
int launch_short(const ShortArgs<T> &a, bool model, cudaStream_t st)
{
    if (a.nbricks <= 0) return MSM_OK;
    const int grid = (a.nbricks + SR_WARPS - 1) / SR_WARPS;
    if (model) k_short<T, true, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    else k_short<T, false, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_count_pairs(const ShortArgs<T> &a, cudaStream_t st)
{
    if (a.nbricks <= 0) return MSM_OK;
    const int grid = (a.nbricks + SR_WARPS - 1) / SR_WARPS;
    k_short<T, false, true><<<grid, SR_WARPS * 32, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_count_pairs<float>(const ShortArgs<float> &, cudaStream_t);
template int launch_count_pairs<double>(const ShortArgs<double> &, cudaStream_t);

template int launch_short<float>(const ShortArgs<float> &, bool, cudaStream_t);
template int launch_short<double>(const ShortArgs<double> &, bool, cudaStream_t);

}  // namespace msm
