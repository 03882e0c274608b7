// k_grid.cu -- the long-range steps of the MSM (Sec. 3):
//   k_anterp       q^0_mu = sum_j phi^0_mu(r_j) q_j, one thread per grid point
//                  gathering the atoms of the 4^3 cells its basis function
//                  touches (cells mu-2 .. mu+1 per axis): no atomics
//   k_restrict     q^{k+1}_mu = sum_nu Phi(nu/2 - mu)^{x3} q^k_nu: taps at
//                  nu - 2mu in {-3,-1,0,1,3} with weights {-1,9,16,9,-1}/16
//   k_stencil      u^{k,cut}_mu = sum_n 2^{-k} W[n] q^k_{mu+n}, W[n] = g^0(|n| h)
//                  for |n| h < 2a (g^k(2^k r) = 2^{-k} g^0(r)): every level
//                  0..l-2 in one launch; shared-memory tile with a halo of
//                  rad points, 4 outputs per thread along x held in registers,
//                  rows of the tap sphere unrolled per half-width
//   k_top          u^{l-1}_mu = sum_nu g^{l-1}(|r_mu - r_nu|) q_nu in FP64 over
//                  a precomputed Toeplitz table (one warp per output point)
//   k_prolong      u^k_mu = u^{k,cut}_mu + sum_nu Phi(mu/2 - nu)^{x3} u^{k+1}_nu
//   k_interp       phi_i = k_e (u_i^short + sum_mu phi^0_mu(r_i) u^0_mu - q_i gamma(0)/a),
//                  F_i = k_e (F_i^short - q_i sum_mu grad phi^0_mu(r_i) u^0_mu) [+ LJ],
//                  scattered back to the caller's atom order
#include "kernels.cuh"

namespace msm {

// ---------------------------------------------------------------- anterpolation

template <int O, typename T> __device__ __forceinline__ T wsel(T f)
{
    // weight of grid point c - 1 + O for an atom at fraction f in cell c
    const T g = T(1) - f;
    if (O == 0) return T(-0.5) * f * g * g;
    if (O == 1) return g * (T(1) + f - T(1.5) * f * f);
    if (O == 2) return f * (T(1) + g - T(1.5) * g * g);
    return T(-0.5) * g * f * f;
}

template <int OZ, int OY, int OX, typename T>
__device__ __forceinline__ void anterp_cell(const int *__restrict__ start, const vec4<T> *__restrict__ afrac,
                                            int cell, T &acc)
{
    const int s0 = start[cell], s1 = start[cell + 1];
    for (int s = s0; s < s1; s++) {
        const vec4<T> f = afrac[s];
        acc = fma(wsel<OZ>(f.z) * wsel<OY>(f.y), wsel<OX>(f.x) * f.w, acc);
    }
}

template <typename T>
__global__ void k_anterp(const AnterpArgs<T> A)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    const LevelGeom &L = A.L0;
    if (idx >= L.n[0] * L.n[1] * L.n[2] || failed(A.status)) return;
    const int ix = idx % L.n[0], iy = (idx / L.n[0]) % L.n[1], iz = idx / (L.n[0] * L.n[1]);
    const int mx = L.lo[0] + ix, my = L.lo[1] + iy, mz = L.lo[2] + iz;
    const int nx = A.cg.nc[0], ny = A.cg.nc[1], nz = A.cg.nc[2];
    T acc = 0;
    // grid point mu receives weight index O = mu - c + 1 from an atom in cell c
#pragma unroll
    for (int oz = 0; oz < 4; oz++) {
        const int cz = mz + 1 - oz;
        if (cz < 0 || cz >= nz) continue;
#pragma unroll
        for (int oy = 0; oy < 4; oy++) {
            const int cy = my + 1 - oy;
            if (cy < 0 || cy >= ny) continue;
            const int rb = (cz * ny + cy) * nx;
#pragma unroll
            for (int ox = 0; ox < 4; ox++) {
                const int cx = mx + 1 - ox;
                if (cx < 0 || cx >= nx) continue;
                const int cell = rb + cx;
#define AC(a, b, c) if (oz == a && oy == b && ox == c) anterp_cell<a, b, c, T>(A.start, A.afrac, cell, acc);
#define AC4(a, b) AC(a, b, 0) AC(a, b, 1) AC(a, b, 2) AC(a, b, 3)
#define AC16(a) AC4(a, 0) AC4(a, 1) AC4(a, 2) AC4(a, 3)
                AC16(0) AC16(1) AC16(2) AC16(3)
#undef AC16
#undef AC4
#undef AC
            }
        }
    }
    A.q0[L.off + idx] = acc;
}

template <typename T>
int launch_anterp(const AnterpArgs<T> &a, cudaStream_t st)
{
    const int m = a.L0.n[0] * a.L0.n[1] * a.L0.n[2];
    k_anterp<T><<<(m + 255) / 256, 256, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
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
__global__ void k_restrict(LevelGeom F, LevelGeom C, const T *__restrict__ qf, T *__restrict__ qc,
                           const int *__restrict__ status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= C.n[0] * C.n[1] * C.n[2] || failed(status)) return;
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
            const T *row = qf + F.off + (size_t)(nz * F.n[1] + ny) * F.n[0];
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
    qc[C.off + idx] = acc;
}

template <typename T>
int launch_restrict(const LevelGeom &fine, const LevelGeom &coarse, const T *qf, T *qc, const int *status,
                    cudaStream_t st)
{
    const int m = coarse.n[0] * coarse.n[1] * coarse.n[2];
    k_restrict<T><<<(m + 255) / 256, 256, 0, st>>>(fine, coarse, qf, qc, status);
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

constexpr int ST_TXT = 8;     // threads along x
constexpr int ST_R = 4;       // outputs per thread along x
constexpr int ST_TY = 4;
constexpr int ST_TZ = 4;
constexpr int ST_TX = ST_TXT * ST_R;
constexpr int ST_THREADS = ST_TXT * ST_TY * ST_TZ;
constexpr int ST_MAXRAD = 12;

__host__ __device__ constexpr int st_sx(int rad) { return ((ST_TX + 2 * rad) | 3) ; }   // odd stride: conflict-free rows
__host__ __device__ constexpr int st_sy(int rad) { return ST_TY + 2 * rad; }
__host__ __device__ constexpr int st_sz(int rad) { return ST_TZ + 2 * rad; }

template <typename T> size_t stencil_smem_bytes(int rad)
{
    return sizeof(T) * (size_t)st_sx(rad) * st_sy(rad) * st_sz(rad);
}
template size_t stencil_smem_bytes<float>(int);
template size_t stencil_smem_bytes<double>(int);

template <int W, typename T>
__device__ __forceinline__ void stencil_row(const T *__restrict__ s, const T *__restrict__ wr, T (&acc)[ST_R])
{
    T v[ST_R + 2 * W];
#pragma unroll
    for (int i = 0; i < ST_R + 2 * W; i++) v[i] = s[i - W];
#pragma unroll
    for (int d = -W; d <= W; d++) {
        const T w = __ldg(wr + d);
#pragma unroll
        for (int r = 0; r < ST_R; r++) acc[r] = fma(w, v[r + d + W], acc[r]);
    }
}

template <typename T>
__global__ void __launch_bounds__(ST_THREADS) k_stencil(const StencilArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *tile = reinterpret_cast<T *>(smem_raw);
    if (failed(A.status)) return;
    int lev = 0;
    while (lev + 1 < A.nlev && (int)blockIdx.x >= A.blk_off[lev + 1]) lev++;
    const int b = blockIdx.x - A.blk_off[lev];
    const LevelGeom &L = A.gg.L[lev];
    const int tx = b % A.tiles[lev][0], ty = (b / A.tiles[lev][0]) % A.tiles[lev][1],
              tz = b / (A.tiles[lev][0] * A.tiles[lev][1]);
    const int x0 = tx * ST_TX, y0 = ty * ST_TY, z0 = tz * ST_TZ;     // tile origin (array indices)
    const int rad = A.sg.rad;
    const int SX = st_sx(rad), SY = st_sy(rad), SZ = st_sz(rad);
    const T *__restrict__ q = A.q + L.off;

    // stage q over the tile plus a halo of rad points (zero outside the grid)
    const int tot = SX * SY * SZ;
    for (int e = threadIdx.x; e < tot; e += ST_THREADS) {
        const int sx = e % SX, sy = (e / SX) % SY, sz = e / (SX * SY);
        const int gx = x0 + sx - rad, gy = y0 + sy - rad, gz = z0 + sz - rad;
        T v = 0;
        if (sx < ST_TX + 2 * rad && gx >= 0 && gx < L.n[0] && gy >= 0 && gy < L.n[1] && gz >= 0 && gz < L.n[2])
            v = q[(size_t)(gz * L.n[1] + gy) * L.n[0] + gx];
        tile[e] = v;
    }
    __syncthreads();

    const int lx = threadIdx.x % ST_TXT, ly = (threadIdx.x / ST_TXT) % ST_TY, lz = threadIdx.x / (ST_TXT * ST_TY);
    T acc[ST_R];
#pragma unroll
    for (int r = 0; r < ST_R; r++) acc[r] = 0;
    const int wd = A.sg.wdim;
    for (int ri = 0; ri < A.sg.nrows; ri++) {
        const int4 row = A.rows[ri];
        const T *s = tile + ((lz + rad + row.y) * SY + (ly + rad + row.x)) * SX + lx * ST_R + rad;
        const T *wr = A.w + ((row.y + rad) * wd + (row.x + rad)) * wd + rad;
        switch (row.z) {
        case 0: stencil_row<0>(s, wr, acc); break;
        case 1: stencil_row<1>(s, wr, acc); break;
        case 2: stencil_row<2>(s, wr, acc); break;
        case 3: stencil_row<3>(s, wr, acc); break;
        case 4: stencil_row<4>(s, wr, acc); break;
        case 5: stencil_row<5>(s, wr, acc); break;
        case 6: stencil_row<6>(s, wr, acc); break;
        case 7: stencil_row<7>(s, wr, acc); break;
        case 8: stencil_row<8>(s, wr, acc); break;
        case 9: stencil_row<9>(s, wr, acc); break;
        case 10: stencil_row<10>(s, wr, acc); break;
        case 11: stencil_row<11>(s, wr, acc); break;
        default: stencil_row<12>(s, wr, acc); break;
        }
    }
    const T scale = (T)ldexp(1.0, -lev);            // g^k = 2^{-k} g^0 at level-k spacing
    const int gy = y0 + ly, gz = z0 + lz;
    if (gy < L.n[1] && gz < L.n[2]) {
        T *out = A.ucut + L.off + (size_t)(gz * L.n[1] + gy) * L.n[0];
#pragma unroll
        for (int r = 0; r < ST_R; r++) {
            const int gx = x0 + lx * ST_R + r;
            if (gx < L.n[0]) out[gx] = scale * acc[r];
        }
    }
}

template <typename T>
int launch_stencil(const StencilArgs<T> &a, cudaStream_t st)
{
    if (a.nlev <= 0) return MSM_OK;
    if (a.sg.rad > ST_MAXRAD) return fail_msg(MSM_EINVAL, "stencil radius %d exceeds %d (2a/h too large)", a.sg.rad, ST_MAXRAD);
    const size_t smem = stencil_smem_bytes<T>(a.sg.rad);
    CUDA_TRY(cudaFuncSetAttribute(k_stencil<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_stencil<T><<<a.blk_off[a.nlev], ST_THREADS, smem, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

void stencil_tiles(const LevelGeom &L, int t[3])
{
    t[0] = (L.n[0] + ST_TX - 1) / ST_TX;
    t[1] = (L.n[1] + ST_TY - 1) / ST_TY;
    t[2] = (L.n[2] + ST_TZ - 1) / ST_TZ;
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
__global__ void k_top(LevelGeom L, const double *__restrict__ table, const T *__restrict__ q,
                      double *__restrict__ u, const int *__restrict__ status)
{
    const int lane = threadIdx.x & 31;
    const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int m = L.n[0] * L.n[1] * L.n[2];
    if (p >= m || failed(status)) return;
    const int px = p % L.n[0], py = (p / L.n[0]) % L.n[1], pz = p / (L.n[0] * L.n[1]);
    const int wx = 2 * L.n[0] - 1, wy = 2 * L.n[1] - 1;
    const T *qt = q + L.off;
    double acc = 0.0;
    for (int j = lane; j < m; j += 32) {
        const int jx = j % L.n[0], jy = (j / L.n[0]) % L.n[1], jz = j / (L.n[0] * L.n[1]);
        const int t = ((pz - jz + L.n[2] - 1) * wy + (py - jy + L.n[1] - 1)) * wx + (px - jx + L.n[0] - 1);
        acc = fma(table[t], (double)qt[j], acc);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) u[p] = acc;
}

template <typename T>
int launch_top(const LevelGeom &top, const double *table, const T *qtop, double *utop, const int *status,
               cudaStream_t st)
{
    const int m = top.n[0] * top.n[1] * top.n[2];
    k_top<T><<<(m * 32 + 255) / 256, 256, 0, st>>>(top, table, qtop, utop, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ---------------------------------------------------------------- prolongation

template <typename T, typename S>
__global__ void k_prolong(LevelGeom F, LevelGeom C, const T *__restrict__ ucut, const S *__restrict__ uc,
                          T *__restrict__ uf, const int *__restrict__ status)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F.n[0] * F.n[1] * F.n[2] || failed(status)) return;
    const int m[3] = {F.lo[0] + idx % F.n[0], F.lo[1] + (idx / F.n[0]) % F.n[1], F.lo[2] + idx / (F.n[0] * F.n[1])};
    int nu0[3], cnt[3];
    T w[3][4];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        if ((m[d] & 1) == 0) {                     // even: only nu = mu/2 (Phi(0) = 1; Phi(+-1) = 0)
            nu0[d] = m[d] >> 1; cnt[d] = 1; w[d][0] = T(1);
        } else {                                   // odd: nu = (mu-3)/2 .. (mu+3)/2
            nu0[d] = (m[d] - 3) >> 1; cnt[d] = 4;
            w[d][0] = T(-1.0 / 16.0); w[d][1] = T(9.0 / 16.0); w[d][2] = T(9.0 / 16.0); w[d][3] = T(-1.0 / 16.0);
        }
    }
    T acc = 0;
    for (int a = 0; a < cnt[2]; a++) {
        const int cz = nu0[2] + a - C.lo[2];
        if (cz < 0 || cz >= C.n[2]) continue;
        for (int b = 0; b < cnt[1]; b++) {
            const int cy = nu0[1] + b - C.lo[1];
            if (cy < 0 || cy >= C.n[1]) continue;
            const T wzy = w[2][a] * w[1][b];
            T racc = 0;
            for (int c = 0; c < cnt[0]; c++) {
                const int cx = nu0[0] + c - C.lo[0];
                if (cx < 0 || cx >= C.n[0]) continue;
                racc = fma(w[0][c], (T)uc[(cz * C.n[1] + cy) * C.n[0] + cx], racc);
            }
            acc = fma(wzy, racc, acc);
        }
    }
    uf[F.off + idx] = ucut[F.off + idx] + acc;
}

template <typename T, typename S>
int launch_prolong(const LevelGeom &fine, const LevelGeom &coarse, const T *ucut, const S *uc, T *uf,
                   const int *status, cudaStream_t st)
{
    const int m = fine.n[0] * fine.n[1] * fine.n[2];
    k_prolong<T, S><<<(m + 255) / 256, 256, 0, st>>>(fine, coarse, ucut, uc, uf, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ---------------------------------------------------------------- interpolation

template <typename T>
__global__ void k_interp(const InterpArgs<T> A)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= A.n || failed(A.status)) return;
    const int key = A.akey[s];
    const int nx = A.cg.nc[0], ny = A.cg.nc[1];
    const int cx = key % nx, cy = (key / nx) % ny, cz = key / (nx * ny);
    const vec4<T> f = A.afrac[s];
    T wx[4], wy[4], wz[4], dx[4], dy[4], dz[4];
    phi_weights_d(f.x, wx, dx);
    phi_weights_d(f.y, wy, dy);
    phi_weights_d(f.z, wz, dz);
    const LevelGeom &L = A.L0;
    // grid point mu = c - 1 + o sits at array index c - 1 + o - lo = c + o (lo = -1)
    const T *u = A.u0 + L.off;
    T p = 0, gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int oz = 0; oz < 4; oz++) {
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
    const vec4<T> sr = A.sr[s];
    const int i = A.perm[s];
    const double q = A.q[i];
    const double ke = A.ke, ih = A.inv_h;
    const double phi = ke * ((double)sr.w + (double)p - q * A.self);
    double F[3] = {ke * ((double)sr.x - q * (double)gx * ih), ke * ((double)sr.y - q * (double)gy * ih),
                   ke * ((double)sr.z - q * (double)gz * ih)};
    double e = 0.5 * q * phi;
    if (A.lj) {
        const vec4<T> lj = A.lj[s];
        F[0] += (double)lj.x; F[1] += (double)lj.y; F[2] += (double)lj.z;
        e += 0.5 * (double)lj.w;
    }
    if (A.wall_k > 0.0) {                          // flat-bottom wall of the water completion
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double x = A.pos[3 * i + d];
            const double lo = A.wall_w - (x - A.box_lo[d]), hi = A.wall_w - (A.box_hi[d] - x);
            if (lo > 0.0) { F[d] += A.wall_k * lo; e += 0.5 * A.wall_k * lo * lo; }
            if (hi > 0.0) { F[d] -= A.wall_k * hi; e += 0.5 * A.wall_k * hi * hi; }
        }
    }
    if (A.forces) { A.forces[3 * i] = F[0]; A.forces[3 * i + 1] = F[1]; A.forces[3 * i + 2] = F[2]; }
    if (A.pot) A.pot[i] = phi;
    A.eatom[i] = e;
    A.vatom[i] = A.pos[3 * i] * F[0] + A.pos[3 * i + 1] * F[1] + A.pos[3 * i + 2] * F[2];
}

template <typename T>
int launch_interp(const InterpArgs<T> &a, cudaStream_t st)
{
    if (a.n <= 0) return MSM_OK;
    k_interp<T><<<(a.n + 255) / 256, 256, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ------------------------------------------------------------ instantiations

template int launch_anterp<float>(const AnterpArgs<float> &, cudaStream_t);
template int launch_anterp<double>(const AnterpArgs<double> &, cudaStream_t);
template int launch_restrict<float>(const LevelGeom &, const LevelGeom &, const float *, float *, const int *, cudaStream_t);
template int launch_restrict<double>(const LevelGeom &, const LevelGeom &, const double *, double *, const int *, cudaStream_t);
template int launch_stencil<float>(const StencilArgs<float> &, cudaStream_t);
template int launch_stencil<double>(const StencilArgs<double> &, cudaStream_t);
template int launch_top<float>(const LevelGeom &, const double *, const float *, double *, const int *, cudaStream_t);
template int launch_top<double>(const LevelGeom &, const double *, const double *, double *, const int *, cudaStream_t);
template int launch_prolong<float, float>(const LevelGeom &, const LevelGeom &, const float *, const float *, float *, const int *, cudaStream_t);
template int launch_prolong<float, double>(const LevelGeom &, const LevelGeom &, const float *, const double *, float *, const int *, cudaStream_t);
template int launch_prolong<double, double>(const LevelGeom &, const LevelGeom &, const double *, const double *, double *, const int *, cudaStream_t);
template int launch_interp<float>(const InterpArgs<float> &, cudaStream_t);
template int launch_interp<double>(const InterpArgs<double> &, cudaStream_t);

}  // namespace msm
