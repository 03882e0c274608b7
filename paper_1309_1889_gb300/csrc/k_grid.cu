// k_grid.cu -- the long-range steps of the MSM (Sec. 3):
//   k_anterp       q^0_mu = sum_j phi^0_mu(r_j) q_j, one thread per column of
//                  4 grid points gathering the atoms of the cells their basis
//                  functions touch (cells mu-2 .. mu+1 per axis): no atomics
//   k_restrict     q^{k+1}_mu = sum_nu Phi(nu/2 - mu)^{x3} q^k_nu: taps at
//                  nu - 2mu in {-3,-1,0,1,3} with weights {-1,9,16,9,-1}/16
//   k_stencil      u^{k,cut}_mu = sum_n 2^{-k} W[n] q^k_{mu+n}, W[n] = g^0(|n| h)
//                  for |n| h < 2a (g^k(2^k r) = 2^{-k} g^0(r)): every level
//                  0..l-2 in one launch; the planes of a tile and its halo of
//                  rad points come into shared memory by TMA (mbarrier-paced
//                  double buffer), 8 x 2 outputs per thread held in registers,
//                  rows of the tap sphere unrolled per half-width
//   k_top          u^{l-1}_mu = sum_nu g^{l-1}(|r_mu - r_nu|) q_nu in FP64 over
//                  a precomputed Toeplitz table (one warp per output point)
//   k_prolong      u^k_mu = u^{k,cut}_mu + sum_nu Phi(mu/2 - nu)^{x3} u^{k+1}_nu
//   k_interp       phi_i = k_e (u_i^short + sum_mu phi^0_mu(r_i) u^0_mu - q_i gamma(0)/a),
//                  F_i = k_e (F_i^short - q_i sum_mu grad phi^0_mu(r_i) u^0_mu) [+ LJ],
//                  scattered back to the caller's atom order (for multiple time
//                  stepping the two terms of F_i as fast and slow forces)
//
// Every kernel serves a batch of systems (one launch per stage for all of
// them): blockIdx.y picks the system for the per-point and per-atom kernels,
// and the persistent lattice-cutoff kernel takes tiles of every (system,
// level) pair from one counter.
#include <algorithm>
#include <cstring>

#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

#include "kernels.cuh"

namespace msm {

// ---------------------------------------------------------------- anterpolation


// A thread owns AN_Z consecutive level-0 points along z at one (x, y); a CTA
// is an AN_X x AN_Y patch of such columns.  Point mu receives, from an atom in
// cell c, the weight with index O = mu - c + 1 per axis (cells mu - 2 .. mu + 1).
// For each of the 4 cell rows in y and the AN_Z + 3 rows in z that reach the
// column, the 4 cells mu_x - 2 .. mu_x + 1 of the row are one contiguous range
// of sorted slots; every atom of it adds (q wx[Ox] wy[Oy]) wz[Oz] to the up to
// 4 points of the column it reaches (Oz fixed by the row, so the accumulator
// of each term is known at compile time).  Weights come precomputed per
// sorted atom (BinArgs::aw).  Each point sums its atoms in a fixed order
// (y rows, then z rows, then slots) whatever the launch shape: no atomics.
constexpr int AN_X = 16, AN_Y = 8, AN_Z = 4;

template <typename T>
__global__ void __launch_bounds__(AN_X * AN_Y) k_anterp(const AnterpArgs<T> A)
{
    if (failed(A.status)) return;
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const LevelGeom &L = D.gg.L[0];
    const int ntx = (L.n[0] + AN_X - 1) / AN_X, nty = (L.n[1] + AN_Y - 1) / AN_Y, ntz = (L.n[2] + AN_Z - 1) / AN_Z;
    if ((int)blockIdx.x >= ntx * nty * ntz) return;
    const int bx = blockIdx.x % ntx, by = (blockIdx.x / ntx) % nty, bz = blockIdx.x / (ntx * nty);
    const int ix = bx * AN_X + threadIdx.x % AN_X, iy = by * AN_Y + threadIdx.x / AN_X, iz0 = bz * AN_Z;
    if (ix >= L.n[0] || iy >= L.n[1]) return;
    const int nx = D.g.nc[0], ny = D.g.nc[1], nz = D.g.nc[2];
    const int mx = L.lo[0] + ix, my = L.lo[1] + iy, mz0 = L.lo[2] + iz0;
    const int *__restrict__ start = A.start + D.cell_off;
    const vec4<T> *__restrict__ wxq = A.aw;
    const T *__restrict__ wy = &A.aw[A.n_total].x;
    const vec4<T> *__restrict__ wz = A.aw + 2 * (size_t)A.n_total;
    int xc[5];                                    // cells mu_x - 2 .. mu_x + 2 clamped to [0, nx]
#pragma unroll
    for (int k = 0; k < 5; k++) xc[k] = min(max(mx - 2 + k, 0), nx);
    T acc[AN_Z];
#pragma unroll
    for (int p = 0; p < AN_Z; p++) acc[p] = T(0);
#pragma unroll 1
    for (int oy = 0; oy < 4; oy++) {
        const int cy = my + 1 - oy;
        if (cy < 0 || cy >= ny) continue;
#pragma unroll
        for (int rz = 0; rz < AN_Z + 3; rz++) {
            const int cz = mz0 - 2 + rz;
            if (cz < 0 || cz >= nz) continue;
            const int rb = (cz * ny + cy) * nx;
            const int b0 = start[rb + xc[0]], b1 = start[rb + xc[1]], b2 = start[rb + xc[2]];
            const int b3 = start[rb + xc[3]], b4 = start[rb + xc[4]];
            for (int s = b0; s < b4; s++) {
                const int ox = 3 - (s >= b1) - (s >= b2) - (s >= b3);
                const T t = (&wxq[s].x)[ox] * wy[4 * (size_t)s + oy];
                const vec4<T> z = wz[s];
                // the point rz - 3 + Oz takes weight wz[Oz]
                if (rz - 3 >= 0 && rz - 3 < AN_Z) acc[rz - 3 >= 0 ? rz - 3 : 0] += t * z.x;
                if (rz - 2 >= 0 && rz - 2 < AN_Z) acc[rz - 2 >= 0 ? rz - 2 : 0] += t * z.y;
                if (rz - 1 >= 0 && rz - 1 < AN_Z) acc[rz - 1 >= 0 ? rz - 1 : 0] += t * z.z;
                if (rz < AN_Z) acc[rz < AN_Z ? rz : 0] += t * z.w;
            }
        }
    }
    T *out = A.q + D.grid_off + L.off + ((size_t)iz0 * L.n[1] + iy) * L.n[0] + ix;
    const size_t plane = (size_t)L.n[1] * L.n[0];
#pragma unroll
    for (int p = 0; p < AN_Z; p++)
        if (iz0 + p < L.n[2]) out[p * plane] = acc[p];
}

template <typename T>
int launch_anterp(const AnterpArgs<T> &a, cudaStream_t st)
{
    if (a.max_tiles <= 0) return MSM_OK;
    k_anterp<T><<<dim3(a.max_tiles, a.bt.B), AN_X * AN_Y, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

int anterp_tiles(const LevelGeom &L)
{
    return ((L.n[0] + AN_X - 1) / AN_X) * ((L.n[1] + AN_Y - 1) / AN_Y) * ((L.n[2] + AN_Z - 1) / AN_Z);
}

// ------------------------------------------------------------------ restriction

__device__ __forceinline__ double rtap(int o)
{
    // Phi(o/2) for o = nu - 2 mu in [-3, 3]
    switch (o < 0 ? -o : o) {
    case 0: return 1.0;
    case 1: return 9.0 / 16.0;
    case 3: return -1.0 / 16.0;
    default: return 0.0;
    }
}

template <typename T>
__global__ void k_restrict(const Batch bt, int k, T *__restrict__ q, const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const LevelGeom &F = D.gg.L[k], &C = D.gg.L[k + 1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C.n[0] * C.n[1] * C.n[2] || failed(status)) return;
    const T *__restrict__ qf = q + D.grid_off + F.off;
    const int mx = C.lo[0] + idx % C.n[0], my = C.lo[1] + (idx / C.n[0]) % C.n[1],
              mz = C.lo[2] + idx / (C.n[0] * C.n[1]);
    const int offs[5] = {-3, -1, 0, 1, 3};
    T acc = 0;
#pragma unroll
    for (int a = 0; a < 5; a++) {
        const int nz = 2 * mz + offs[a] - F.lo[2];
        if (nz < 0 || nz >= F.n[2]) continue;
        const T wz = (T)rtap(offs[a]);
#pragma unroll
        for (int b = 0; b < 5; b++) {
            const int ny = 2 * my + offs[b] - F.lo[1];
            if (ny < 0 || ny >= F.n[1]) continue;
            const T wy = wz * (T)rtap(offs[b]);
            const T *row = qf + (size_t)(nz * F.n[1] + ny) * F.n[0];
            T racc = 0;
#pragma unroll
            for (int c = 0; c < 5; c++) {
                const int nx = 2 * mx + offs[c] - F.lo[0];
                if (nx < 0 || nx >= F.n[0]) continue;
                racc = fma((T)rtap(offs[c]), row[nx], racc);
            }
            acc = fma(wy, racc, acc);
        }
    }
    q[D.grid_off + C.off + idx] = acc;
}

template <typename T>
int launch_restrict(const Batch &bt, int k, int max_coarse, T *q, const int *status, cudaStream_t st)
{
    if (max_coarse <= 0) return MSM_OK;
    k_restrict<T><<<dim3((max_coarse + 255) / 256, bt.B), 256, 0, st>>>(bt, k, q, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ------------------------------------------------------------ lattice cutoff

// Smoothing gamma and the level-0 kernel in FP64 (used only to build tables).
__device__ __forceinline__ double gamma64(double rho)
{
    if (rho < 1.0) { const double r2 = rho * rho; return GAMMA_C0 + GAMMA_C1 * r2 + GAMMA_C2 * r2 * r2; }
    return 1.0 / rho;
}

__global__ void k_stencil_table(double a, double h, int rad, double *__restrict__ w)
{
    const int wd = 2 * rad + 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= wd * wd * wd) return;
    const int dx = idx % wd - rad, dy = (idx / wd) % wd - rad, dz = idx / (wd * wd) - rad;
    const double r = sqrt((double)(dx * dx + dy * dy + dz * dz)) * h;
    double v = 0.0;
    if (r < 2.0 * a) v = gamma64(r / a) / a - gamma64(r / (2.0 * a)) / (2.0 * a);   // g^0(r)
    w[idx] = v;
}

int launch_stencil_table(double a, double h, int rad, double *wd, cudaStream_t st)
{
    const int m = (2 * rad + 1) * (2 * rad + 1) * (2 * rad + 1);
    k_stencil_table<<<(m + 255) / 256, 256, 0, st>>>(a, h, rad, wd);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Lattice cutoff, all levels 0..l-2 in one persistent launch.  A thread owns
// ST_RX outputs along x times ST_RZ along z in registers.  The ST_NT threads of
// a CTA cover TGX = min(ceil(n_x / ST_RX), ST_MAXGX) groups along x times
// TYR = ST_NT / TGX rows along y, so a tile spans whole grid rows of short
// levels (the 100-point level-0 rows of a 23.5 nm box waste 6 % of the
// threads, fixed 32-point tiles 23 %).  The tile's input planes z' = z0-rad ..
// z0+ST_RZ-1+rad come into two shared-memory buffers by TMA: one thread
// starts a cp.async.bulk.tensor copy of the plane's box (the tile's rows with
// their halos; the hardware fills points outside the grid with zeros) on the
// buffer's mbarrier, the next plane's copy in flight while the current one is
// used.  The box starts on a 16-byte boundary in x (the halo is rounded up to
// whole groups of 4 values) and its width is an odd number of 16-byte granules
// (consecutive rows fall in different banks).  The plane rows y + dy and y - dy
// (the weights depend on |dy|) are added once in registers and applied to the
// ST_RZ output planes they reach (dz = z' - z), walking the tap row (|dy|, |dz|)
// of the sphere with compile-time offsets: half the multiply-adds of walking
// every row.  The weights W[n] = g^0(|n| h) depend on |n| only, so one octant of
// the table sits in shared memory; the level factor 2^{-k} is applied at the
// end.  A tile's input planes are split in two halves (the first rad + ST_RZ/2
// planes and the rest), taken by two CTAs: twice the warps per SM to hide the
// shared-load latency, with no extra plane traffic.  Each half adds its scaled
// partial sum into the zeroed output by an atomic add; with exactly two addends
// onto zero the result does not depend on which lands first (IEEE addition
// commutes).  CTAs take tile halves from a counter.  Each half sums its taps in
// a fixed order (planes, row pairs, then x offsets), whatever the tile shape.
constexpr int ST_RX = 8, ST_RZ = 2, ST_NT = 128, ST_MAXGX = 16;
constexpr int ST_SPLIT = 2;         // plane halves per tile (two addends: order-free)
constexpr int ST_MAXRAD = 12;
constexpr int ST_MAXMAPS = 24;      // descriptors per launch (kernel parameter: 24 x 128 bytes)
constexpr long ST_WAIT_POLLS = 1L << 22;

struct StTile { int tgx, tyr, ntx, nty, ntz; };
__host__ __device__ inline StTile st_tile(const LevelGeom &L)
{
    StTile t;
    const int nxg = (L.n[0] + ST_RX - 1) / ST_RX;
    t.tgx = nxg < ST_MAXGX ? nxg : ST_MAXGX;
    t.tyr = ST_NT / t.tgx;
    t.ntx = (nxg + t.tgx - 1) / t.tgx;
    t.nty = (L.n[1] + t.tyr - 1) / t.tyr;
    t.ntz = (L.n[2] + ST_RZ - 1) / ST_RZ;
    return t;
}

// Rows of values are handled in groups of 4 (16 bytes of FP32).
__host__ __device__ constexpr int st_up4(int v) { return (v + 3) & ~3; }
__host__ __device__ constexpr int st_r1p(int rad) { return st_up4(rad + 1); }
// x halo of a tile, rounded up to whole groups: the box starts on a 16-byte boundary
__host__ __device__ constexpr int st_radp(int rad) { return st_up4(rad); }
// box width: the tile's x range and both halos, an odd number of groups of 4 values
__host__ __device__ inline int st_bx(int tgx, int rad)
{
    int g = (tgx * ST_RX + 2 * st_radp(rad)) / 4;
    if (!(g & 1)) g++;
    return 4 * g;
}
// box height: the tile's rows and both halos
__host__ __device__ inline int st_by(int tgx, int rad) { return ST_NT / tgx + 2 * rad; }

// Shared memory of one CTA: 128 bytes of alignment slack, the weight octant
// W[|dz|][|dy|][|dx|] ((rad+1)^2 rows of st_r1p values) rounded up to 128
// bytes, two plane buffers of `plane` values (a multiple of 32 values: both
// buffers start on 128-byte boundaries), and the half-widths of the tap rows by
// (|dz|, |dy|).
__host__ __device__ inline size_t st_up128(size_t b) { return (b + 127) & ~(size_t)127; }
template <typename T> size_t stencil_smem_bytes(int rad, int plane)
{
    const size_t r1 = (size_t)rad + 1;
    return 128 + st_up128(sizeof(T) * r1 * r1 * (size_t)st_r1p(rad)) + sizeof(T) * 2 * (size_t)plane +
           sizeof(int) * (r1 * r1 + 4);
}
template size_t stencil_smem_bytes<float>(int, int);
template size_t stencil_smem_bytes<double>(int, int);

int stencil_plane_values(const LevelGeom &L, int rad)
{
    const StTile t = st_tile(L);
    return (st_bx(t.tgx, rad) * st_by(t.tgx, rad) + 31) & ~31;
}

// Values of one plane row in registers: ST_RX + 2 st_radp(RAD).
template <int RAD> struct StRow { static constexpr int N = st_up4(ST_RX + 2 * st_radp(RAD)); };

// acc[r] += sum_{|d| <= W} w[|d|] v[r + d + st_radp(RAD)]; w: the octant row |dx| = 0..RAD of
// the tap row, already in registers (loaded with the plane rows, before the switch on W)
template <int RAD> struct StW { static constexpr int N = st_r1p(RAD); };

template <int W, int RAD, typename T>
__device__ __forceinline__ void stencil_row(const T (&v)[StRow<RAD>::N], const T (&w)[StW<RAD>::N], T (&acc)[ST_RX])
{
    constexpr int RP = st_radp(RAD);
#pragma unroll
    for (int d = -W; d <= W; d++) {
#pragma unroll
        for (int r = 0; r < ST_RX; r++) acc[r] = fma(w[d < 0 ? -d : d], v[r + d + RP], acc[r]);
    }
}

template <int RAD, typename T>
__device__ __forceinline__ void stencil_row_dispatch(int w, const T (&v)[StRow<RAD>::N], const T (&wr)[StW<RAD>::N],
                                                     T (&acc)[ST_RX])
{
    switch (w) {
#define ST_CASE(k) case k: if (k <= RAD) stencil_row<(k <= RAD ? k : 0), RAD>(v, wr, acc); break;
    ST_CASE(0) ST_CASE(1) ST_CASE(2) ST_CASE(3) ST_CASE(4) ST_CASE(5) ST_CASE(6)
    ST_CASE(7) ST_CASE(8) ST_CASE(9) ST_CASE(10) ST_CASE(11) ST_CASE(12)
#undef ST_CASE
    default: break;
    }
}

// A weight row (st_r1p values, 16-byte aligned) from shared memory into registers.
template <int RAD, typename T>
__device__ __forceinline__ void st_load_w(const T *__restrict__ wr, T (&w)[StW<RAD>::N])
{
    if (sizeof(T) == sizeof(float)) {
#pragma unroll
        for (int k = 0; k < StW<RAD>::N; k += 4) {
            const float4 f = *reinterpret_cast<const float4 *>(wr + k);
            w[k] = f.x; w[k + 1] = f.y; w[k + 2] = f.z; w[k + 3] = f.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < StW<RAD>::N; k++) w[k] = wr[k];
    }
}

// The descriptors of one launch: entries e0 .. e0+ne-1 of the batch.
struct StMaps {
    CUtensorMap map[ST_MAXMAPS];
    int e0, ne;
};

__device__ __forceinline__ uint32_t st_smem(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Start the TMA copy of the box at (x, y, z) into dst; the barrier expects its bytes.
__device__ __forceinline__ void st_tma_plane(const CUtensorMap *map, void *dst, uint64_t *bar, int x, int y, int z,
                                             uint32_t bytes)
{
    const uint32_t b = st_smem(bar), d = st_smem(dst);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
                 ::"r"(d), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(b)
                 : "memory");
}

// Wait for the barrier phase with the given parity: at most ST_WAIT_POLLS polls.
__device__ __forceinline__ bool st_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t b = st_smem(bar);
    for (long i = 0; i < ST_WAIT_POLLS; i++) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(b), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

template <typename T, int RAD>
__global__ void __launch_bounds__(ST_NT) k_stencil(const __grid_constant__ StencilArgs<T> A,
                                                   const __grid_constant__ StMaps M, int *__restrict__ counter)
{
    constexpr int WD = 2 * RAD + 1, R1 = RAD + 1, R1P = st_r1p(RAD), RP = st_radp(RAD);
    extern __shared__ unsigned char smem_raw[];
    const int PLANE = A.sg.plane;
    unsigned char *base = smem_raw + ((128 - (st_smem(smem_raw) & 127)) & 127);
    T *wt = reinterpret_cast<T *>(base);                     // R1 x R1 rows of R1P weights W[|dz|][|dy|][|dx|]
    T *buf0 = reinterpret_cast<T *>(base + st_up128(sizeof(T) * R1 * R1 * R1P));   // two plane buffers
    int *hw = reinterpret_cast<int *>(buf0 + 2 * PLANE);     // R1^2 half widths by (|dz|, |dy|) (-1: empty)
    __shared__ __align__(8) uint64_t bars[2];
    __shared__ int s_tile, s_ent, s_err;
    if (failed(A.status)) return;
    const int t = threadIdx.x;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(st_smem(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(st_smem(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        s_err = 0;
    }
    for (int e = t; e < R1 * R1 * R1P; e += ST_NT) {
        const int ax = e % R1P, ay = (e / R1P) % R1, az = e / (R1P * R1);
        wt[e] = ax < R1 ? A.w[((az + RAD) * WD + (ay + RAD)) * WD + (ax + RAD)] : T(0);
    }
    for (int e = t; e < R1 * R1; e += ST_NT) hw[e] = -1;
    __syncthreads();
    for (int e = t; e < A.sg.nrows; e += ST_NT) {
        const int4 r = A.rows[e];
        if (r.x >= 0 && r.y >= 0) hw[r.y * R1 + r.x] = r.z;
    }
    uint32_t phase[2] = {0u, 0u};                            // the barriers' next phases (uniform)
    const int e_end = M.e0 + M.ne;
    const int first = A.blk_off[M.e0], total = A.blk_off[e_end];
    for (;;) {
        __syncthreads();
        if (t == 0) {
            const int tile = first + atomicAdd(counter, 1);
            // owner (system, level) of the tile: last entry whose first tile is <= tile
            int lo_e = M.e0, hi_e = e_end - 1;
            while (lo_e < hi_e) {
                const int mid = (lo_e + hi_e + 1) >> 1;
                if (A.blk_off[mid] <= tile) lo_e = mid; else hi_e = mid - 1;
            }
            s_tile = tile;
            s_ent = lo_e;
        }
        __syncthreads();
        const int tile = s_tile;
        if (tile >= total) break;
        const int ent = s_ent, lev = ent % A.nlev;
        const SysDesc &D = A.bt.sd[ent / A.nlev];
        const LevelGeom &L = D.gg.L[lev];
        const StTile tg = st_tile(L);
        const int PX = st_bx(tg.tgx, RAD);
        const uint32_t bytes = (uint32_t)(sizeof(T) * PX * st_by(tg.tgx, RAD));
        const CUtensorMap *map = &M.map[ent - M.e0];
        const int part = (tile - A.blk_off[ent]) % ST_SPLIT, b = (tile - A.blk_off[ent]) / ST_SPLIT;
        const int tx = b % tg.ntx, ty = (b / tg.ntx) % tg.nty, tz = b / (tg.ntx * tg.nty);
        const int x0 = tx * tg.tgx * ST_RX, y0 = ty * tg.tyr, z0 = tz * ST_RZ;
        // A 16-byte shared load of a warp is served eight lanes at a time.  Eight
        // consecutive lanes take eight consecutive rows of one x group: the box
        // width is an odd number of 16-byte granules, so their row loads fall in
        // different banks.  The tyr % 8 rows left over per x group come last, two
        // rows of four x groups per eight lanes when two are left (distinct banks
        // again).  Which thread owns an output changes nothing in its sum.
        const int full = tg.tyr & ~7, rem = tg.tyr - full, nblk = (full >> 3) * tg.tgx;
        int yr, xg;
        if (t < 8 * nblk) {
            xg = (t >> 3) % tg.tgx;
            yr = ((t >> 3) / tg.tgx) * 8 + (t & 7);
        } else if (rem > 0) {
            xg = (t - 8 * nblk) / rem;
            yr = full + (t - 8 * nblk) % rem;
        } else {
            xg = tg.tgx;
            yr = 0;
        }
        const bool active = xg < tg.tgx;
        const int ny = L.n[1], nz = L.n[2];
        // this half's planes that exist: z' in [zb, ze)
        constexpr int ZH = RAD + ST_RZ / 2;
        const int zlo = z0 - RAD + part * ZH, zhi = part == ST_SPLIT - 1 ? z0 + ST_RZ + RAD : zlo + ZH;
        const int zb = max(zlo, 0), ze = min(zhi, nz);
        T acc[ST_RZ][ST_RX];
#pragma unroll
        for (int s = 0; s < ST_RZ; s++)
#pragma unroll
            for (int r = 0; r < ST_RX; r++) acc[s][r] = 0;
        if (t == 0 && zb < ze) st_tma_plane(map, buf0, &bars[0], x0 - RP, y0 - RAD, zb, bytes);
        for (int zp = zb; zp < ze; zp++) {
            const int bi = (zp - zb) & 1;
            T *cur = buf0 + bi * PLANE;
            // the other buffer was last read in the previous plane, before its closing barrier
            if (t == 0 && zp + 1 < ze)
                st_tma_plane(map, buf0 + (bi ^ 1) * PLANE, &bars[bi ^ 1], x0 - RP, y0 - RAD, zp + 1, bytes);
            if (!st_wait(&bars[bi], phase[bi])) s_err = 1;
            __syncthreads();
            if (s_err) {
                // a copy that did not arrive: report, give the copies in flight a bounded
                // wait of their own, leave (every thread of the CTA takes this branch)
                if (t == 0) set_status(const_cast<int *>(A.status), MSM_ETIMEOUT);
                st_wait(&bars[bi], phase[bi]);
                if (zp + 1 < ze) st_wait(&bars[bi ^ 1], phase[bi ^ 1]);
                return;
            }
            phase[bi] ^= 1u;
            if (active) {
                // W depends on |dy|: rows y + dy and y - dy are added once and share
                // the tap row of (|dz|, |dy|) for both output planes.  Every shared-memory
                // read of an iteration (the two half-widths, the two weight rows, the two
                // plane rows) is issued before the first multiply-add needs one of them.
                int adz_s[ST_RZ];
                bool on_s[ST_RZ];
#pragma unroll
                for (int s = 0; s < ST_RZ; s++) {
                    const int dz = zp - (z0 + s);
                    on_s[s] = dz >= -RAD && dz <= RAD;
                    adz_s[s] = on_s[s] ? (dz < 0 ? -dz : dz) : 0;
                }
#pragma unroll 1
                for (int ady = 0; ady <= RAD; ady++) {
                    constexpr int NV = StRow<RAD>::N;
                    int wsel[ST_RZ];
                    T wrow[ST_RZ][StW<RAD>::N];
#pragma unroll
                    for (int s = 0; s < ST_RZ; s++) {
                        wsel[s] = on_s[s] ? hw[adz_s[s] * R1 + ady] : -1;
                        st_load_w<RAD>(wt + (adz_s[s] * R1 + ady) * R1P, wrow[s]);
                    }
                    T v[NV];
                    const T *row = cur + (yr + RAD + ady) * PX + xg * ST_RX;      // 16-byte aligned
                    const T *mir = cur + (yr + RAD - ady) * PX + xg * ST_RX;
                    if (sizeof(T) == sizeof(float)) {
#pragma unroll
                        for (int i = 0; i < NV; i += 4) {
                            const float4 f = *reinterpret_cast<const float4 *>(row + i);
                            v[i] = f.x; v[i + 1] = f.y; v[i + 2] = f.z; v[i + 3] = f.w;
                        }
                        if (ady > 0) {
#pragma unroll
                            for (int i = 0; i < NV; i += 4) {
                                const float4 f = *reinterpret_cast<const float4 *>(mir + i);
                                v[i] += f.x; v[i + 1] += f.y; v[i + 2] += f.z; v[i + 3] += f.w;
                            }
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < NV; i++) v[i] = ady > 0 ? row[i] + mir[i] : row[i];
                    }
#pragma unroll
                    for (int s = 0; s < ST_RZ; s++)
                        if (wsel[s] >= 0) stencil_row_dispatch<RAD>(wsel[s], v, wrow[s], acc[s]);
                }
            }
            __syncthreads();                          // the buffer is refilled two planes on
        }
        const T scale = (T)ldexp(1.0, -lev);        // g^k = 2^{-k} g^0 at level-k spacing
        const int gy = y0 + yr;
        if (active && gy < ny) {
#pragma unroll
            for (int s = 0; s < ST_RZ; s++) {
                const int gz = z0 + s;
                if (gz >= nz) continue;
                T *out = A.ucut + D.grid_off + L.off + ((size_t)gz * ny + gy) * L.n[0];
#pragma unroll
                for (int r = 0; r < ST_RX; r++) {
                    const int gx = x0 + xg * ST_RX + r;
                    if (gx < L.n[0]) atomicAdd(out + gx, scale * acc[s][r]);
                }
            }
        }
    }
}

// cuTensorMapEncodeTiled from the driver, through the runtime's entry-point lookup.
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

template <typename T>
int encode_stencil_maps(const SysDesc *sd, int B, int nlev, int rad, const T *q, CUtensorMap *maps)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail_msg(MSM_ECUDA, "cuTensorMapEncodeTiled is not available");
    for (int s = 0; s < B; s++)
        for (int k = 0; k < nlev; k++) {
            const SysDesc &D = sd[s];
            const LevelGeom &L = D.gg.L[k];
            const StTile tg = st_tile(L);
            const T *base = q + D.grid_off + L.off;
            if ((reinterpret_cast<uintptr_t>(base) & 15) || (L.n[0] * sizeof(T)) % 16)
                return fail_msg(MSM_EINVAL, "lattice-cutoff grid rows are not 16-byte aligned");
            const cuuint64_t dims[3] = {(cuuint64_t)L.n[0], (cuuint64_t)L.n[1], (cuuint64_t)L.n[2]};
            const cuuint64_t strides[2] = {(cuuint64_t)L.n[0] * sizeof(T), (cuuint64_t)L.n[0] * L.n[1] * sizeof(T)};
            const cuuint32_t box[3] = {(cuuint32_t)st_bx(tg.tgx, rad), (cuuint32_t)st_by(tg.tgx, rad), 1u};
            const cuuint32_t estr[3] = {1u, 1u, 1u};
            const CUresult r = enc(&maps[(size_t)s * nlev + k],
                                   sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                   3, const_cast<T *>(base), dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                return fail_msg(MSM_ECUDA, "cuTensorMapEncodeTiled failed (%d) for system %d, level %d", (int)r, s, k);
        }
    return MSM_OK;
}
template int encode_stencil_maps<float>(const SysDesc *, int, int, int, const float *, CUtensorMap *);
template int encode_stencil_maps<double>(const SysDesc *, int, int, int, const double *, CUtensorMap *);

template <typename T, int RAD>
static int launch_stencil_rad(const StencilArgs<T> &a, const CUtensorMap *maps, const int *blk, int *counter,
                              int sms, cudaStream_t st)
{
    const size_t smem = stencil_smem_bytes<T>(RAD, a.sg.plane);
    CUDA_TRY(cudaFuncSetAttribute(k_stencil<T, RAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stencil<T, RAD>, ST_NT, smem));
    if (per_sm < 1) return fail_msg(MSM_EINVAL, "lattice-cutoff tile does not fit (radius %d)", RAD);
    const int nent = a.bt.B * a.nlev;
    CUDA_TRY(cudaMemsetAsync(a.ucut, 0, sizeof(T) * a.ucut_len, st));
    for (int e0 = 0; e0 < nent; e0 += ST_MAXMAPS) {
        StMaps m;
        m.e0 = e0;
        m.ne = std::min(ST_MAXMAPS, nent - e0);
        memcpy(m.map, maps + e0, sizeof(CUtensorMap) * (size_t)m.ne);
        const int tiles = blk[e0 + m.ne] - blk[e0];
        if (tiles <= 0) continue;
        CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), st));
        const int grid = std::min(tiles, sms * per_sm);
        k_stencil<T, RAD><<<grid, ST_NT, smem, st>>>(a, m, counter);
        count_launch();
        CUDA_TRY(cudaGetLastError());
    }
    return MSM_OK;
}

template <typename T>
int launch_stencil(const StencilArgs<T> &a, const CUtensorMap *maps, const int *blk, int *counter, cudaStream_t st)
{
    if (a.nlev <= 0 || a.total_tiles <= 0) return MSM_OK;
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    switch (a.sg.rad) {
#define ST_RADCASE(r) case r: return launch_stencil_rad<T, r>(a, maps, blk, counter, sms, st);
    ST_RADCASE(1) ST_RADCASE(2) ST_RADCASE(3) ST_RADCASE(4) ST_RADCASE(5) ST_RADCASE(6)
    ST_RADCASE(7) ST_RADCASE(8) ST_RADCASE(9) ST_RADCASE(10) ST_RADCASE(11) ST_RADCASE(12)
#undef ST_RADCASE
    default: return fail_msg(MSM_EINVAL, "lattice-cutoff radius %d outside 1..%d", a.sg.rad, ST_MAXRAD);
    }
}

int stencil_tile_count(const LevelGeom &L)
{
    const StTile t = st_tile(L);
    return t.ntx * t.nty * t.ntz * ST_SPLIT;
}

// ------------------------------------------------------------------ top level

__global__ void k_top_table(LevelGeom L, double a_top, double h_top, double *__restrict__ t)
{
    const int wx = 2 * L.n[0] - 1, wy = 2 * L.n[1] - 1, wz = 2 * L.n[2] - 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= wx * wy * wz) return;
    const int dx = idx % wx - (L.n[0] - 1), dy = (idx / wx) % wy - (L.n[1] - 1), dz = idx / (wx * wy) - (L.n[2] - 1);
    const double r = sqrt((double)dx * dx + (double)dy * dy + (double)dz * dz) * h_top;
    t[idx] = gamma64(r / a_top) / a_top;           // g^{l-1}(r) = gamma(r / 2^{l-1} a) / (2^{l-1} a)
}

int launch_top_table(const LevelGeom &top, double a_top, double h_top, double *table, cudaStream_t st)
{
    const int m = (2 * top.n[0] - 1) * (2 * top.n[1] - 1) * (2 * top.n[2] - 1);
    k_top_table<<<(m + 255) / 256, 256, 0, st>>>(top, a_top, h_top, table);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
__global__ void k_top(const Batch bt, const double *__restrict__ table, const T *__restrict__ q,
                      double *__restrict__ u, const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const LevelGeom &L = D.gg.L[D.gg.levels - 1];
    const int lane = threadIdx.x & 31;
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int m = L.n[0] * L.n[1] * L.n[2];
    if (p >= m || failed(status)) return;
    const int px = p % L.n[0], py = (p / L.n[0]) % L.n[1], pz = p / (L.n[0] * L.n[1]);
    const int wx = 2 * L.n[0] - 1, wy = 2 * L.n[1] - 1;
    const T *qt = q + D.grid_off + L.off;
    const double *tab = table + D.ttab_off;
    double acc = 0.0;
    for (int j = lane; j < m; j += 32) {
        const int jx = j % L.n[0], jy = (j / L.n[0]) % L.n[1], jz = j / (L.n[0] * L.n[1]);
        const int t = ((pz - jz + L.n[2] - 1) * wy + (py - jy + L.n[1] - 1)) * wx + (px - jx + L.n[0] - 1);
        acc = fma(tab[t], (double)qt[j], acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[D.top_off + p] = acc;
}

template <typename T>
int launch_top(const Batch &bt, int max_top, const double *table, const T *q, double *utop, const int *status,
               cudaStream_t st)
{
    if (max_top <= 0) return MSM_OK;
    k_top<T><<<dim3((max_top * 32 + 255) / 256, bt.B), 256, 0, st>>>(bt, table, q, utop, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
__global__ void k_top_to_grid(const Batch bt, const double *__restrict__ utop, T *__restrict__ u,
                              const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const LevelGeom &L = D.gg.L[D.gg.levels - 1];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= L.n[0] * L.n[1] * L.n[2] || failed(status)) return;
    u[D.grid_off + L.off + p] = (T)utop[D.top_off + p];
}

template <typename T>
int launch_top_to_grid(const Batch &bt, int max_top, const double *utop, T *u, const int *status, cudaStream_t st)
{
    if (max_top <= 0) return MSM_OK;
    k_top_to_grid<T><<<dim3((max_top + 255) / 256, bt.B), 256, 0, st>>>(bt, utop, u, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ---------------------------------------------------------------- prolongation

template <typename T, typename S>
__device__ __forceinline__ T prolong_point(const LevelGeom &F, const LevelGeom &C, int idx, const S *__restrict__ uc)
{
    const int m[3] = {F.lo[0] + idx % F.n[0], F.lo[1] + (idx / F.n[0]) % F.n[1], F.lo[2] + idx / (F.n[0] * F.n[1])};
    // Four coarse points per axis nu0 .. nu0+3 with weights Phi(mu/2 - nu):
    // even mu: nu0 = mu/2 - 1, weights (0, 1, 0, 0); odd mu: nu0 = (mu-3)/2, weights (-1, 9, 9, -1)/16.
    int c0[3];
    T w[3][4];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const bool odd = m[d] & 1;
        c0[d] = (odd ? (m[d] - 3) >> 1 : (m[d] >> 1) - 1) - C.lo[d];
        w[d][0] = odd ? T(-1.0 / 16.0) : T(0);
        w[d][1] = odd ? T(9.0 / 16.0) : T(1);
        w[d][2] = odd ? T(9.0 / 16.0) : T(0);
        w[d][3] = odd ? T(-1.0 / 16.0) : T(0);
    }
    T acc = 0;
#pragma unroll
    for (int a = 0; a < 4; a++) {
        const int cz = c0[2] + a;
        if (w[2][a] == T(0) || cz < 0 || cz >= C.n[2]) continue;
#pragma unroll
        for (int b = 0; b < 4; b++) {
            const int cy = c0[1] + b;
            if (w[1][b] == T(0) || cy < 0 || cy >= C.n[1]) continue;
            const S *row = uc + (size_t)(cz * C.n[1] + cy) * C.n[0];
            T racc = 0;
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int cx = c0[0] + c;
                if (w[0][c] != T(0) && cx >= 0 && cx < C.n[0]) racc = fma(w[0][c], (T)row[cx], racc);
            }
            acc = fma(w[2][a] * w[1][b], racc, acc);
        }
    }
    return acc;
}

// u^k_mu = u^{k,cut}_mu + prolongation of u^{k+1}; from_top: level k+1 is the
// top level, read in FP64 from the top buffer.
template <typename T>
__global__ void k_prolong(const Batch bt, int k, const T *__restrict__ ucut, const double *__restrict__ utop,
                          bool from_top, T *__restrict__ u, const int *__restrict__ status)
{
    const SysDesc &D = bt.sd[blockIdx.y];
    const LevelGeom &F = D.gg.L[k], &C = D.gg.L[k + 1];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F.n[0] * F.n[1] * F.n[2] || failed(status)) return;
    const T acc = from_top ? prolong_point<T, double>(F, C, idx, utop + D.top_off)
                           : prolong_point<T, T>(F, C, idx, u + D.grid_off + C.off);
    const int o = D.grid_off + F.off + idx;
    u[o] = ucut[o] + acc;
}

template <typename T>
int launch_prolong(const Batch &bt, int k, int max_fine, const T *ucut, const double *utop, bool from_top, T *u,
                   const int *status, cudaStream_t st)
{
    if (max_fine <= 0) return MSM_OK;
    k_prolong<T><<<dim3((max_fine + 255) / 256, bt.B), 256, 0, st>>>(bt, k, ucut, utop, from_top, u, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ---------------------------------------------------------------- interpolation

template <typename T>
__global__ void k_interp(const InterpArgs<T> A)
{
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int ls = blockIdx.x * blockDim.x + threadIdx.x;
    if (ls >= D.n || failed(A.status)) return;
    const int s = D.atom_off + ls;
    const int key = A.akey[s] - D.cell_off;
    const int nx = D.g.nc[0], ny = D.g.nc[1];
    const int cx = key % nx, cy = (key / nx) % ny, cz = key / (nx * ny);
    const vec4<T> f = A.afrac[s];
    T wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    phi_weights_d(f.x, wx, dx);
    phi_weights_d(f.y, wy, dy);
    phi_weights_d(f.z, wz, dz);
    const LevelGeom &L = D.gg.L[0];
    T p = 0, gx = 0, gy = 0, gz = 0;
    // grid point mu = c - 1 + o sits at array index c - 1 + o - lo = c + o (lo = -1);
    // no grids (u = NULL): the cutoff methods, whose pair sums are the whole result
    const T *u = A.u ? A.u + D.grid_off + L.off : nullptr;
#pragma unroll
    for (int oz = 0; u && oz < 4; oz++) {
#pragma unroll
        for (int oy = 0; oy < 4; oy++) {
            const T *row = u + (size_t)((cz + oz) * L.n[1] + (cy + oy)) * L.n[0] + cx;
            T rp = 0, rd = 0;
#pragma unroll
            for (int ox = 0; ox < 4; ox++) {
                const T v = row[ox];
                rp = fma(wx[ox], v, rp);
                rd = fma(dx[ox], v, rd);
            }
            const T wzy = wz[oz] * wy[oy];
            p = fma(wzy, rp, p);
            gx = fma(wzy, rd, gx);
            gy = fma(wz[oz] * dy[oy], rp, gy);
            gz = fma(dz[oz] * wy[oy], rp, gz);
        }
    }
    // Forces combined per atom in T, then one conversion to the FP64 outputs (on the
    // integer pipe: GB300 runs FP64 instructions at 1/64 of the FP32 rate).  The
    // potential and energy are combined in FP64 (a handful of FP64 operations per
    // atom): the grid potential carries each atom's own smooth self-interaction,
    // removed here by q_i gamma(0)/a, and for molecules this nearly cancels against
    // the excluded pairs' smooth terms (FP64 in k_exclusions); an FP32 k_e or self
    // coefficient would round alike for every atom and bias U far beyond 1e-6.
    const int i = A.perm[s];
    const vec4<T> sr = A.sr[i];
    const T q = to_t<T>(A.q[i]);
    const T ke = to_t<T>(A.ke), ih = to_t<T>(D.inv_h);
    // split evaluation (multiple time stepping): F holds the fast part, Fs the grid part
    const bool split = A.fslow != nullptr;
    T F[3], Fs[3] = {T(0), T(0), T(0)};
    if (split) {
        const T kq = ke * q * ih;
        F[0] = ke * sr.x; F[1] = ke * sr.y; F[2] = ke * sr.z;
        Fs[0] = -(kq * gx); Fs[1] = -(kq * gy); Fs[2] = -(kq * gz);
    } else {
        F[0] = ke * (sr.x - q * gx * ih); F[1] = ke * (sr.y - q * gy * ih); F[2] = ke * (sr.z - q * gz * ih);
    }
    const double qd = A.q[i];
    const double phid = A.ke * ((to_d(sr.w) + to_d(p)) - qd * A.self);
    double ed = (0.5 * qd) * phid;
    if (A.lj) {
        const vec4<T> lj = A.lj[i];
        F[0] += lj.x; F[1] += lj.y; F[2] += lj.z;
        ed = fma(0.5, to_d(lj.w), ed);
    }
    double Fd[3] = {to_d(F[0]), to_d(F[1]), to_d(F[2])};
    const double x[3] = {A.pos[3 * i], A.pos[3 * i + 1], A.pos[3 * i + 2]};
    const int c[3] = {cx, cy, cz};
    if (A.wall_k > 0.0 && (c[0] < D.wall_lo[0] || c[0] > D.wall_hi[0] || c[1] < D.wall_lo[1] ||
                           c[1] > D.wall_hi[1] || c[2] < D.wall_lo[2] || c[2] > D.wall_hi[2])) {
        // flat-bottom wall of the water completion (FP64; only cells near a face can reach it)
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double lo = A.wall_w - (x[d] - D.box_lo[d]), hi = A.wall_w - (D.box_hi[d] - x[d]);
            if (lo > 0.0) { Fd[d] += A.wall_k * lo; ed += 0.5 * A.wall_k * lo * lo; }
            if (hi > 0.0) { Fd[d] -= A.wall_k * hi; ed += 0.5 * A.wall_k * hi * hi; }
        }
    }
    if (A.forces) { A.forces[3 * i] = Fd[0]; A.forces[3 * i + 1] = Fd[1]; A.forces[3 * i + 2] = Fd[2]; }
    if (A.pot) A.pot[i] = phid;
    A.eatom[i] = ed;
    if (split) {
        const double Fsd[3] = {to_d(Fs[0]), to_d(Fs[1]), to_d(Fs[2])};
        A.fslow[3 * i] = Fsd[0]; A.fslow[3 * i + 1] = Fsd[1]; A.fslow[3 * i + 2] = Fsd[2];
        A.eslow[i] = (0.5 * qd) * (A.ke * (to_d(p) - qd * A.self));
#pragma unroll
        for (int d = 0; d < 3; d++) Fd[d] += Fsd[d];
    }
    A.vatom[i] = x[0] * Fd[0] + x[1] * Fd[1] + x[2] * Fd[2];
}

template <typename T>
int launch_interp(const InterpArgs<T> &a, cudaStream_t st)
{
    if (a.max_n <= 0) return MSM_OK;
    k_interp<T><<<dim3((a.max_n + 255) / 256, a.bt.B), 256, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ------------------------------------------------------------ instantiations

template int launch_anterp<float>(const AnterpArgs<float> &, cudaStream_t);
template int launch_anterp<double>(const AnterpArgs<double> &, cudaStream_t);
template int launch_restrict<float>(const Batch &, int, int, float *, const int *, cudaStream_t);
template int launch_restrict<double>(const Batch &, int, int, double *, const int *, cudaStream_t);
template int launch_stencil<float>(const StencilArgs<float> &, const CUtensorMap *, const int *, int *,
                                   cudaStream_t);
template int launch_stencil<double>(const StencilArgs<double> &, const CUtensorMap *, const int *, int *,
                                    cudaStream_t);
template int launch_top<float>(const Batch &, int, const double *, const float *, double *, const int *, cudaStream_t);
template int launch_top<double>(const Batch &, int, const double *, const double *, double *, const int *, cudaStream_t);
template int launch_top_to_grid<float>(const Batch &, int, const double *, float *, const int *, cudaStream_t);
template int launch_top_to_grid<double>(const Batch &, int, const double *, double *, const int *, cudaStream_t);
template int launch_prolong<float>(const Batch &, int, int, const float *, const double *, bool, float *, const int *, cudaStream_t);
template int launch_prolong<double>(const Batch &, int, int, const double *, const double *, bool, double *, const int *, cudaStream_t);
template int launch_interp<float>(const InterpArgs<float> &, cudaStream_t);
template int launch_interp<double>(const InterpArgs<double> &, cudaStream_t);

}  // namespace msm
