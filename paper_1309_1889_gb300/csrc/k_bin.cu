// k_bin.cu -- bit-exact cell binning and the stable counting sort of atoms
// by finest-grid cell: the cell lists behind the short-range sum and the
// gather-form anterpolation and interpolation of Sec. 3.
//
//   k_bin_keys     cell of every atom: t = (x - x0) * (1/h) with one IEEE FP64
//                  subtract and one IEEE FP64 multiply (no contraction), c =
//                  floor(t); key = (cz*ny + cy)*nx + cx; histogram by integer
//                  atomics (exact).  Also writes the compute-type copies of
//                  the box-relative position and of the in-cell fraction
//                  t - c (exact in FP64 by Sterbenz) in original order, so no
//                  later kernel repeats FP64 work.
//   k_scan_*       exclusive prefix sum of the histogram -> cell_start
//   k_scatter      atom -> a slot of its cell (order inside a cell arbitrary)
//   k_sort_cells   each cell's slots reordered by atom index: the result is the
//                  unique stable order (key, index), whatever the atomics did
//   k_gather       sorted copies of position, fraction, key and (molecule, LJ)
//                  flag, and each atom's anterpolation weights
//
// A batch of systems is binned by one pass of each kernel: a system's cell ids
// are offset by the cells of the systems before it, so the one global stable
// sort leaves each system's atoms in a contiguous slot range, ordered exactly
// as a sort of that system alone.
#include "kernels.cuh"

namespace msm {

template <typename T>
__global__ void k_bin_keys(const Batch bt, const double *__restrict__ pos, const double *__restrict__ q,
                           int *__restrict__ key, int *__restrict__ count, vec4<T> *__restrict__ rel,
                           vec4<T> *__restrict__ frac, int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= D.n) return;
    const int i = D.atom_off + li;
    const CellGeom &g = D.g;
    int c[3];
    double r[3], f[3];
    // FP64 arithmetic only where the binning contract needs it (the subtract and
    // the multiply, and t - floor(t)); the finiteness and range tests, the floor
    // and the conversions to T act on the IEEE 754 bit fields (GB300 runs FP64
    // instructions at 1/64 of the FP32 rate).
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double x = pos[3 * i + d];
        if (((__double_as_longlong(x) >> 52) & 0x7ff) == 0x7ff) { set_status(status, MSM_EINVAL); key[i] = -1; return; }
        const double rl = __dsub_rn(x, g.origin[d]);
        const double t = __dmul_rn(rl, D.inv_h);
        // floor(t) for 0 <= t < 2^31: clear the fraction bits below the binary point
        const unsigned long long b = (unsigned long long)__double_as_longlong(t);
        const int e = (int)((b >> 52) & 0x7ff) - 1023;                 // unbiased exponent
        if ((b >> 63) && t != 0.0) { set_status(status, MSM_ERANGE); key[i] = -1; return; }   // t < 0
        if (e >= 31) { set_status(status, MSM_ERANGE); key[i] = -1; return; }
        int ci = 0;
        double fl = __longlong_as_double((long long)(b & 0x8000000000000000ull));   // floor of [+-0, 1): signed 0
        if (e >= 0) {
            const int sh = 52 - e;                                      // fraction bits below the point
            ci = (int)((((b & 0xfffffffffffffull) | (1ull << 52))) >> sh);
            fl = __longlong_as_double((long long)(b & ~((1ull << sh) - 1ull)));
        }
        if (ci > g.nc[d] - 1) { set_status(status, MSM_ERANGE); key[i] = -1; return; }
        c[d] = ci;
        r[d] = rl;
        f[d] = __dsub_rn(t, fl);
    }
    int k = D.cell_off + (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    key[i] = k;
    atomicAdd(&count[k], 1);
    T qi = to_t<T>(q[i]);
    rel[i] = vec4<T>{to_t<T>(r[0]), to_t<T>(r[1]), to_t<T>(r[2]), qi};
    frac[i] = vec4<T>{to_t<T>(f[0]), to_t<T>(f[1]), to_t<T>(f[2]), qi};
}

// Exclusive scan in three passes: per-block sums, scan of block sums, add.
constexpr int SCAN_T = 512, SCAN_E = 8, SCAN_B = SCAN_T * SCAN_E;

__device__ __forceinline__ int block_excl_scan(int v, int *tot)
{
    __shared__ int ws[SCAN_T / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < SCAN_T / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, s, o); if (lane >= o) s += y; }
        if (lane < SCAN_T / 32) ws[lane] = s;
    }
    __syncthreads();
    int base = w ? ws[w - 1] : 0;
    *tot = ws[SCAN_T / 32 - 1];
    int r = base + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(int m, const int *__restrict__ in, int *__restrict__ out,
                                                        int *__restrict__ bsum, const int *__restrict__ status)
{
    if (failed(status)) return;
    int b0 = blockIdx.x * SCAN_B + threadIdx.x * SCAN_E;
    int v[SCAN_E], s = 0;
#pragma unroll
    for (int e = 0; e < SCAN_E; e++) { v[e] = (b0 + e < m) ? in[b0 + e] : 0; s += v[e]; }
    int tot;
    int ex = block_excl_scan(s, &tot);
#pragma unroll
    for (int e = 0; e < SCAN_E; e++) { if (b0 + e < m) out[b0 + e] = ex; ex += v[e]; }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block scans the nb block sums in chunks of SCAN_B with a running carry
// (any nb), and writes the grand total.
__global__ void __launch_bounds__(SCAN_T) k_scan_sums(int nb, int *__restrict__ bsum, int *__restrict__ total,
                                                      const int *__restrict__ status)
{
    if (failed(status)) return;
    int carry = 0;
    for (int c0 = 0; c0 < nb; c0 += SCAN_B) {
        const int b0 = c0 + threadIdx.x * SCAN_E;
        int v[SCAN_E], s = 0;
#pragma unroll
        for (int e = 0; e < SCAN_E; e++) { v[e] = (b0 + e < nb) ? bsum[b0 + e] : 0; s += v[e]; }
        int tot;
        int ex = block_excl_scan(s, &tot) + carry;
#pragma unroll
        for (int e = 0; e < SCAN_E; e++) { if (b0 + e < nb) bsum[b0 + e] = ex; ex += v[e]; }
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int m, int *__restrict__ out, const int *__restrict__ bsum, const int *__restrict__ total,
                           const int *__restrict__ status)
{
    if (failed(status)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) out[i] += bsum[i / SCAN_B];
    if (i == 0) out[m] = *total;
}

__global__ void k_scatter(int n, const int *__restrict__ key, const int *__restrict__ start, int *__restrict__ count,
                          int *__restrict__ perm, const int *__restrict__ status)
{
    if (failed(status)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int k = key[i];
    int slot = start[k] + atomicSub(&count[k], 1) - 1;
    perm[slot] = i;
}

__global__ void k_sort_cells(int ncells, const int *__restrict__ start, int *__restrict__ perm,
                             const int *__restrict__ status)
{
    if (failed(status)) return;
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    int s0 = start[c], s1 = start[c + 1];
    for (int s = s0 + 1; s < s1; s++) {           // insertion sort: a cell holds a few atoms
        int v = perm[s], t = s - 1;
        while (t >= s0 && perm[t] > v) { perm[t + 1] = perm[t]; t--; }
        perm[t + 1] = v;
    }
}

// Sorted slots of system s are [atom_off, atom_off + n): its cells come before
// the next system's and every atom lands in a cell of its own system.
template <typename T>
__global__ void k_gather(const Batch bt, int n_total, const int *__restrict__ perm, const int *__restrict__ key,
                         const vec4<T> *__restrict__ rel, const vec4<T> *__restrict__ frac,
                         const uint8_t *__restrict__ lj, vec4<T> *__restrict__ apos,
                         vec4<T> *__restrict__ afrac, int *__restrict__ akey, int *__restrict__ aflag,
                         vec4<T> *__restrict__ aw, const int *__restrict__ status)
{
    if (failed(status)) return;
    const SysDesc &D = bt.sd[blockIdx.y];
    const int ls = blockIdx.x * blockDim.x + threadIdx.x;
    if (ls >= D.n) return;
    const int s = D.atom_off + ls;
    const int i = perm[s];
    apos[s] = rel[i];
    const vec4<T> f = frac[i];
    afrac[s] = f;
    akey[s] = key[i];
    if (aw) {                      // the atom's anterpolation weights (Sec. 3, p = 3), x scaled by q
        T wx[4], wy[4], wz[4];
        phi_weights(f.x, wx);
        phi_weights(f.y, wy);
        phi_weights(f.z, wz);
        aw[s] = vec4<T>{wx[0] * f.w, wx[1] * f.w, wx[2] * f.w, wx[3] * f.w};
        aw[n_total + s] = vec4<T>{wy[0], wy[1], wy[2], wy[3]};
        aw[2 * n_total + s] = vec4<T>{wz[0], wz[1], wz[2], wz[3]};
    }
    const int li = i - D.atom_off;
    const int mol = li < 3 * D.n_mol ? i - li % 3 : i;       // first atom of the molecule; single sites: own
    aflag[s] = (mol << 1) | ((lj && lj[i]) ? 1 : 0);
}

// The integer-pipe binary64 <-> binary32 conversions of the FP32 kernels, on
// device arrays (a diagnostic entry point checks them against the hardware's).
__global__ void k_diag_convert(int64_t n, const double *__restrict__ x, float *__restrict__ x32,
                               const float *__restrict__ y, double *__restrict__ y64)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x32[i] = f32_of(x[i]);
    y64[i] = f64_of(y[i]);
}

int launch_diag_convert(int64_t n, const double *x, float *x32, const float *y, double *y64, cudaStream_t st)
{
    if (n <= 0) return MSM_OK;
    if (n > ((int64_t)1 << 40)) return fail_msg(MSM_EINVAL, "n too large");
    k_diag_convert<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, x32, y, y64);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// block sums of a scan of m values, plus the total
int scan_scratch_ints(int m) { return (m + SCAN_B - 1) / SCAN_B + 2; }

// start[0..m] = exclusive prefix sums of count[0..m-1] (start[m] = total).
int launch_scan(int m, const int *count, int *start, int *bsum, const int *status, cudaStream_t st)
{
    const int nb = (m + SCAN_B - 1) / SCAN_B;
    k_scan_blocks<<<nb, SCAN_T, 0, st>>>(m, count, start, bsum, status);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(nb, bsum, bsum + nb, status);
    k_scan_add<<<(m + 255) / 256, 256, 0, st>>>(m, start, bsum, bsum + nb, status);
    count_launch(3);
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Scan, scatter and per-cell sort of precomputed keys whose histogram is
// already in count[0..m-1]: the second half of launch_bin, for callers that
// compute the keys themselves.
int launch_sort_by_key(int n, int m, const int *key, int *count, int *start, int *perm, int *bsum, int *status,
                       cudaStream_t st)
{
    const int nb = (m + SCAN_B - 1) / SCAN_B;
    k_scan_blocks<<<nb, SCAN_T, 0, st>>>(m, count, start, bsum, status);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(nb, bsum, bsum + nb, status);
    k_scan_add<<<(m + 255) / 256, 256, 0, st>>>(m, start, bsum, bsum + nb, status);
    count_launch(3);
    if (n > 0) {
        k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, key, start, count, perm, status);
        k_sort_cells<<<(m + 255) / 256, 256, 0, st>>>(m, start, perm, status);
        count_launch(2);
    }
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_bin(const BinArgs<T> &a, cudaStream_t st)
{
    const int n = a.n_total, m = a.m_total, B = a.bt.B;
    const int nb = (m + SCAN_B - 1) / SCAN_B;
    CUDA_TRY(cudaMemsetAsync(a.count, 0, sizeof(int) * (size_t)(m + 1), st));
    const dim3 ga((a.max_n + 255) / 256, B);
    if (n > 0) {
        k_bin_keys<T><<<ga, 256, 0, st>>>(a.bt, a.pos, a.q, a.key, a.count, a.rel, a.frac, a.status);
        count_launch();
    }
    k_scan_blocks<<<nb, SCAN_T, 0, st>>>(m, a.count, a.start, a.bsum, a.status);
    k_scan_sums<<<1, SCAN_T, 0, st>>>(nb, a.bsum, a.bsum + nb, a.status);
    k_scan_add<<<(m + 255) / 256, 256, 0, st>>>(m, a.start, a.bsum, a.bsum + nb, a.status);
    count_launch(3);
    if (n > 0) {
        k_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, a.key, a.start, a.count, a.perm, a.status);
        k_sort_cells<<<(m + 255) / 256, 256, 0, st>>>(m, a.start, a.perm, a.status);
        k_gather<T><<<ga, 256, 0, st>>>(a.bt, n, a.perm, a.key, a.rel, a.frac, a.lj, a.apos, a.afrac, a.akey,
                                        a.aflag, a.aw, a.status);
        count_launch(3);
    }
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_bin<float>(const BinArgs<float> &, cudaStream_t);
template int launch_bin<double>(const BinArgs<double> &, cudaStream_t);

}  // namespace msm
