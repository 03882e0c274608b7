// k_md.cu -- everything around the MSM evaluation on the MD path:
//   k_exclusions   rigid-water completion: the short-range kernel skipped the
//                  three intramolecular pairs of each (O, H, H) triple, so only
//                  their smooth part k_e q_i q_j gamma(r/a)/a, which the grids
//                  carry, is subtracted here (forces in T, energy and
//                  potentials in FP64); together this removes the full 1/r =
//                  g* + gamma(r/a)/a of every excluded pair
//   k_sum_*        deterministic FP64 sums (fixed partition, fixed tree) for
//                  the energy, the virial and the kinetic energy
//   k_vv_first     velocity Verlet (Sec. 2): half kick, drift, then SHAKE
//                  for each rigid triple (one thread per molecule)
//   k_vv_second    second half kick, RATTLE velocity stage, kinetic energy
//   k_pr_update    parareal correction lambda^{k+1}_{n+1} = F + (G_new - G_old)
//                  in FP64 (Sec. 4) with the max |dx| partials
//   k_record_uk    (U, K) of every system after a step, at a step index kept
//                  on the device so that a replayed CUDA graph writes each
//                  step's entry
//   k_add          y += x (multiple time stepping: fast + slow forces)
//
// The per-system kernels take a batch: blockIdx.y is the system.
#include "kernels.cuh"

namespace msm {

// ---------------------------------------------------------------- exclusions

template <typename T>
__global__ void k_exclusions(const ExclArgs A)
{
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int mo = blockIdx.x * blockDim.x + threadIdx.x;
    if (mo >= D.n_mol || failed(A.status)) return;
    const int i0 = D.atom_off + 3 * mo;
    // bond vectors from two FP64 differences against the O atom, then T
    T rel[3][3], q[3], F[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        q[a] = to_t<T>(A.q[i0 + a]);
#pragma unroll
        for (int d = 0; d < 3; d++) {
            rel[a][d] = a ? to_t<T>(A.x[3 * (i0 + a) + d] - A.x[3 * i0 + d]) : T(0);
            F[a][d] = 0;
        }
    }
    const T ke = to_t<T>(A.ke), ia = to_t<T>(A.inv_a);
    // The energy and potential terms are formed in FP64.  Per molecule they cancel the
    // atoms' self terms q_i^2 gamma(0)/a (also FP64, in k_interp) to a small remainder
    // (a neutral molecule's own smooth field nearly vanishes at its atoms), while each
    // is ~1e2 kJ/mol; an FP32 k_e, 1/a or gamma would round alike for every molecule of
    // the rigid model and leave a bias of ~1e-7 of that sum: ~1e-5 of U for water.
    const double kd = A.ke * A.inv_a, ia2 = A.inv_a * A.inv_a;
    double qd[3], dphid[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 3; a++) qd[a] = A.q[i0 + a];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int a = c == 2 ? 1 : 0, b = c == 0 ? 1 : 2;
        const T dx = rel[a][0] - rel[b][0], dy = rel[a][1] - rel[b][1], dz = rel[a][2] - rel[b][2];
        const T r2t = dx * dx + dy * dy + dz * dz;
        const T r = sqrt(r2t);
        const T rho = r * ia;
        T dgam;                                        // gamma'(rho)
        const double rho2 = to_d(r2t) * ia2;
        double gam;                                    // gamma(rho), FP64
        if (rho2 < 1.0) {
            gam = GAMMA_C0 + rho2 * (GAMMA_C1 + GAMMA_C2 * rho2);
            dgam = T(2 * GAMMA_C1) * rho + T(4 * GAMMA_C2) * (rho * rho) * rho;
        } else {
            gam = 1.0 / sqrt(rho2);
            const T g = T(1) / rho;
            dgam = -g * g;
        }
        const double kg = kd * gam;                    // k_e gamma(r/a)/a: smooth part of k_e/r
        dphid[a] = fma(-kg, qd[b], dphid[a]);
        dphid[b] = fma(-kg, qd[a], dphid[b]);
        // U_corr = -k_e q_a q_b gamma(r/a)/a  =>  F_a = k_e q_a q_b gamma'(r/a)/a^2 (r_a - r_b)/r
        const T s = ke * q[a] * q[b] * dgam * ia * ia / r;
        F[a][0] += s * dx; F[a][1] += s * dy; F[a][2] += s * dz;
        F[b][0] -= s * dx; F[b][1] -= s * dy; F[b][2] -= s * dz;
    }
    // split evaluation (multiple time stepping): the correction is smooth, a part of the slow force
    double *fout = A.fslow ? A.fslow : A.forces;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int i = i0 + a;
        double v = 0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double fd = to_d(F[a][d]);
            if (fout) fout[3 * i + d] += fd;
            v += A.x[3 * i + d] * fd;
        }
        if (A.pot) A.pot[i] += dphid[a];
        A.eatom[i] += 0.5 * qd[a] * dphid[a];          // each pair's -1/2 e to both atoms
        if (A.eslow) A.eslow[i] += 0.5 * qd[a] * dphid[a];
        A.vatom[i] += v;
    }
}

template <typename T>
int launch_exclusions(const ExclArgs &a, cudaStream_t st)
{
    if (a.max_mol <= 0) return MSM_OK;
    k_exclusions<T><<<dim3((a.max_mol + 127) / 128, a.bt.B), 128, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}
template int launch_exclusions<float>(const ExclArgs &, cudaStream_t);
template int launch_exclusions<double>(const ExclArgs &, cudaStream_t);

// ---------------------------------------------------------------- FP64 sums

constexpr int SUM_T = 256;
constexpr int SUM_CHUNK = 4096;    // values per block: fixed partition

__host__ __device__ int sum_blocks(int n) { return n > 0 ? (n + SUM_CHUNK - 1) / SUM_CHUNK : 1; }

__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double ws[SUM_T / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) ws[w] = v;
    __syncthreads();
    double r = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < SUM_T / 32; k++) r += ws[k];
    __syncthreads();
    return r;
}

struct SumCols { const double *c[4]; };

// block (x, s): chunk x of system s
__global__ void k_sum_partials(const Batch bt, int ncols, SumCols cols, double *__restrict__ part, int total_blocks,
                               const int *__restrict__ status)
{
    if (status && failed(status)) return;
    const SysDesc &D = bt.sd[blockIdx.y];
    if ((int)blockIdx.x >= sum_blocks(D.n)) return;
    const int b0 = blockIdx.x * SUM_CHUNK, e0 = min(D.n, b0 + SUM_CHUNK);
    for (int c = 0; c < ncols; c++) {
        const double *col = cols.c[c] + D.atom_off;
        double v = 0;
        for (int i = b0 + threadIdx.x; i < e0; i += SUM_T) v += col[i];
        v = block_sum(v);
        if (threadIdx.x == 0) part[c * total_blocks + D.part_off + blockIdx.x] = v;
    }
}

// block s: the partials of system s in order
__global__ void k_sum_final(const Batch bt, int ncols, const double *__restrict__ part, int total_blocks,
                            double *__restrict__ out, int out_stride, const int *__restrict__ status)
{
    if (status && failed(status)) return;
    const SysDesc &D = bt.sd[blockIdx.x];
    const int nblk = sum_blocks(D.n);
    for (int c = 0; c < ncols; c++) {
        double v = 0;
        for (int i = threadIdx.x; i < nblk; i += SUM_T) v += part[c * total_blocks + D.part_off + i];
        v = block_sum(v);
        if (threadIdx.x == 0) out[blockIdx.x * out_stride + c] = v;
    }
}

int launch_sum(const Batch &bt, int max_n, int total_blocks, int ncols, const double *const *cols, double *part,
               double *out, int out_stride, const int *status, cudaStream_t st)
{
    if (ncols > 4) return fail_msg(MSM_EINVAL, "launch_sum: at most 4 columns");
    SumCols sc;
    for (int c = 0; c < 4; c++) sc.c[c] = c < ncols ? cols[c] : nullptr;
    k_sum_partials<<<dim3(sum_blocks(max_n), bt.B), SUM_T, 0, st>>>(bt, ncols, sc, part, total_blocks, status);
    k_sum_final<<<bt.B, SUM_T, 0, st>>>(bt, ncols, part, total_blocks, out, out_stride, status);
    count_launch(2);
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// --------------------------------------------------------- velocity Verlet

// Bond c of a triple joins atoms (0,1), (0,2), (1,2): compile-time tables.
__device__ __forceinline__ constexpr int bond_i(int c) { return c == 2 ? 1 : 0; }
__device__ __forceinline__ constexpr int bond_j(int c) { return c == 0 ? 1 : 2; }

// One thread per molecule (or single site), VV_T per CTA.  The CTA's molecules
// are 9 consecutive doubles each in x, v and f: they are staged through shared
// memory with coalesced loads and stores (a thread reading its own 9 values
// from global memory touches 18 cache lines per warp-wide load).
constexpr int VV_T = 128;

template <typename T>
__global__ void __launch_bounds__(VV_T) k_vv_first(const VVArgs A)
{
    __shared__ double sx[VV_T * 9], sv[VV_T * 9], sf[VV_T * 9];
    __shared__ int s_failed;
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int units = D.n_mol + (D.n - 3 * D.n_mol);
    const int u0 = blockIdx.x * VV_T;
    if (u0 >= units) return;
    if (threadIdx.x == 0) s_failed = failed(A.status);
    __syncthreads();
    if (s_failed) return;
    const int u = u0 + threadIdx.x;
    const double dt = A.dt;
    const int nmb = max(0, min(VV_T, D.n_mol - u0));              // molecules of this CTA
    const size_t g0 = 3 * ((size_t)D.atom_off + 3 * (size_t)u0);   // their first double
    for (int e = threadIdx.x; e < 9 * nmb; e += VV_T) {
        const double x = A.x[g0 + e];
        sx[e] = x;
        A.xo[g0 + e] = x;                                          // positions before the drift
        sv[e] = A.v[g0 + e];
        sf[e] = A.fs ? A.f[g0 + e] + A.ws * A.fs[g0 + e] : A.f[g0 + e];
    }
    __syncthreads();
    if (u < D.n_mol) {
        // The state stays FP64; what a step adds to it (half kick, drift, SHAKE
        // correction) is formed in T in molecule-local coordinates (relative to
        // the old O position), so x and v take one FP64 add per component.
        // GB300 runs FP64 instructions at 1/64 of the FP32 rate: the conversions
        // use the integer pipe, and no FP64 value is kept live across the SHAKE
        // loop (holding 18 doubles through it cost ~11 FP64-pipe instructions per
        // iteration); the state is read again from shared memory after it.
        const int b = 9 * threadIdx.x, i0 = D.atom_off + 3 * u;
        const T tdt = (T)dt, hk = (T)(0.5 * dt), inv_dt = T(1) / tdt;
        T p[3][3], p0[3][3], ro[3][3], w[3], d2[3];
        {
            T rel[3][3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                w[a] = to_t<T>(A.im[i0 + a]);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int k = b + 3 * a + d;
                    rel[a][d] = a ? to_t<T>(sx[k] - sx[b + d]) : T(0);
                    const T dv = hk * to_t<T>(sf[k]) * w[a];                          // half kick
                    p0[a][d] = p[a][d] = rel[a][d] + tdt * (to_t<T>(sv[k]) + dv);    // drift
                }
            }
#pragma unroll
            for (int c = 0; c < 3; c++)
#pragma unroll
                for (int d = 0; d < 3; d++) ro[c][d] = rel[bond_i(c)][d] - rel[bond_j(c)][d];
        }
        // SHAKE on the drifted local positions p; the old bond vectors ro give the directions
        d2[0] = d2[1] = (T)A.d_oh2;
        d2[2] = (T)A.d_hh2;
        const T tol = (T)A.tol;
        bool ok = false;
        for (int it = 0; it < A.max_iter && !ok; it++) {
            ok = true;
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int a = bond_i(c), bb = bond_j(c);
                T rn[3], rn2 = 0, dot = 0;
#pragma unroll
                for (int d = 0; d < 3; d++) { rn[d] = p[a][d] - p[bb][d]; rn2 += rn[d] * rn[d]; }
                const T diff = d2[c] - rn2;
                if ((diff < T(0) ? -diff : diff) > tol * d2[c]) {
                    ok = false;
#pragma unroll
                    for (int d = 0; d < 3; d++) dot += ro[c][d] * rn[d];
                    const T g = diff / (T(2) * dot * (w[a] + w[bb]));
#pragma unroll
                    for (int d = 0; d < 3; d++) { p[a][d] += g * w[a] * ro[c][d]; p[bb][d] -= g * w[bb] * ro[c][d]; }
                }
            }
        }
        if (!ok) { set_status(A.status, MSM_ENOCONV); atomicCAS(A.status + 1, 0, 1); atomicCAS(A.status + 3, 0, i0 + 1); }
        // x = x_old + (drift + dp), v = v_old + (kick + dp / dt): the same kick and
        // drift arithmetic as above, on values read again (volatile: the compiler
        // would otherwise keep the first reads live through the loop)
        const volatile double *vx = sx, *vv = sv, *vf = sf;
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const int k = b + 3 * a + d;
                const double x = vx[k], v = vv[k];
                const T dv = hk * to_t<T>(vf[k]) * w[a];
                const T sd = tdt * (to_t<T>(v) + dv);
                const T dp = p[a][d] - p0[a][d];
                sx[k] = x + to_d(sd + dp);
                sv[k] = v + to_d(dv + dp * inv_dt);
            }
    } else if (u < units) {                                        // single site: half kick, drift
        const int i = D.atom_off + 3 * D.n_mol + (u - D.n_mol);
        const double im = A.im[i];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double x = A.x[3 * i + d];
            const double f = A.fs ? A.f[3 * i + d] + A.ws * A.fs[3 * i + d] : A.f[3 * i + d];
            const double v = A.v[3 * i + d] + 0.5 * dt * f * im;
            A.xo[3 * i + d] = x;
            A.x[3 * i + d] = x + dt * v;
            A.v[3 * i + d] = v;
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * nmb; e += VV_T) {
        A.x[g0 + e] = sx[e];
        A.v[g0 + e] = sv[e];
    }
}

template <typename T>
__global__ void __launch_bounds__(VV_T) k_vv_second(const VVArgs A, double *__restrict__ kin)
{
    __shared__ double sx[VV_T * 9], sv[VV_T * 9], sf[VV_T * 9];
    __shared__ int s_failed;
    const SysDesc &D = A.bt.sd[blockIdx.y];
    const int units = D.n_mol + (D.n - 3 * D.n_mol);
    const int u0 = blockIdx.x * VV_T;
    if (u0 >= units) return;
    if (threadIdx.x == 0) s_failed = failed(A.status);
    __syncthreads();
    if (s_failed) return;
    const int u = u0 + threadIdx.x;
    const double hdt = 0.5 * A.dt;
    const int nmb = max(0, min(VV_T, D.n_mol - u0));
    const size_t g0 = 3 * ((size_t)D.atom_off + 3 * (size_t)u0);
    for (int e = threadIdx.x; e < 9 * nmb; e += VV_T) {
        sx[e] = A.x[g0 + e];
        sv[e] = A.v[g0 + e];
        sf[e] = A.fs ? A.f[g0 + e] + A.ws * A.fs[g0 + e] : A.f[g0 + e];
    }
    __syncthreads();
    if (u < D.n_mol) {
        // as in k_vv_first: the kick and the RATTLE correction form one increment
        // in T, integer-pipe conversions, no FP64 value live across the loop
        const int b = 9 * threadIdx.x, i0 = D.atom_off + 3 * u;
        const T hk = (T)hdt;
        T r[3][3], r2[3], wv[3][3], wm[3];
        {
            T rel[3][3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                wm[a] = to_t<T>(A.im[i0 + a]);
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    const int k = b + 3 * a + d;
                    wv[a][d] = to_t<T>(sv[k]) + hk * to_t<T>(sf[k]) * wm[a];
                    rel[a][d] = a ? to_t<T>(sx[k] - sx[b + d]) : T(0);
                }
            }
            // RATTLE velocity stage: zero the bond-parallel relative velocities
#pragma unroll
            for (int c = 0; c < 3; c++) {
                r2[c] = 0;
#pragma unroll
                for (int d = 0; d < 3; d++) {
                    r[c][d] = rel[bond_i(c)][d] - rel[bond_j(c)][d];
                    r2[c] += r[c][d] * r[c][d];
                }
            }
        }
        const T tol = (T)A.tol_v;
        bool ok = false;
        for (int it = 0; it < A.max_iter && !ok; it++) {
            ok = true;
            // FP64: |rv| <= tol (absolute, as the oracle).  FP32: |rv| <= tol |r| (|v_a| + |v_b|):
            // the rounding of rv = r.(v_a - v_b) grows with the atoms' speeds (not with their
            // difference, which can be tiny), so an absolute or |v_a - v_b|-relative test can stall
            T spd[3];
#pragma unroll
            for (int a = 0; a < 3; a++)
                spd[a] = sizeof(T) == 4 ? sqrt(wv[a][0] * wv[a][0] + wv[a][1] * wv[a][1] + wv[a][2] * wv[a][2]) : T(0);
#pragma unroll
            for (int c = 0; c < 3; c++) {
                const int a = bond_i(c), bb = bond_j(c);
                T rv = 0;
#pragma unroll
                for (int d = 0; d < 3; d++) rv += r[c][d] * (wv[a][d] - wv[bb][d]);
                const T lim = sizeof(T) == 4 ? tol * sqrt(r2[c]) * (spd[a] + spd[bb]) : tol;
                if ((rv < T(0) ? -rv : rv) > lim) {
                    ok = false;
                    const T k = rv / (r2[c] * (wm[a] + wm[bb]));
#pragma unroll
                    for (int d = 0; d < 3; d++) { wv[a][d] -= k * wm[a] * r[c][d]; wv[bb][d] += k * wm[bb] * r[c][d]; }
                }
            }
        }
        if (!ok) { set_status(A.status, MSM_ENOCONV); atomicCAS(A.status + 1, 0, 2); atomicCAS(A.status + 3, 0, i0 + 1); }
        const volatile double *vv = sv;            // read again, not kept through the loop
#pragma unroll
        for (int a = 0; a < 3; a++) {
            double k2 = 0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const int k = b + 3 * a + d;
                const double v = vv[k];
                const double vv = v + to_d(wv[a][d] - to_t<T>(v));
                sv[k] = vv;
                k2 += vv * vv;
            }
            if (kin) kin[i0 + a] = 0.5 * A.m[i0 + a] * k2;
        }
    } else if (u < units) {
        const int i = D.atom_off + 3 * D.n_mol + (u - D.n_mol);
        const double m = A.m[i], im = A.im[i];
        double k2 = 0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double f = A.fs ? A.f[3 * i + d] + A.ws * A.fs[3 * i + d] : A.f[3 * i + d];
            const double v = A.v[3 * i + d] + hdt * f * im;
            A.v[3 * i + d] = v;
            k2 += v * v;
        }
        if (kin) kin[i] = 0.5 * m * k2;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 9 * nmb; e += VV_T) A.v[g0 + e] = sv[e];
}

template <typename T>
int launch_vv_first(const VVArgs &a, cudaStream_t st)
{
    if (a.max_units <= 0) return MSM_OK;
    k_vv_first<T><<<dim3((a.max_units + VV_T - 1) / VV_T, a.bt.B), VV_T, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_vv_second(const VVArgs &a, double *kin_atom, cudaStream_t st)
{
    if (a.max_units <= 0) return MSM_OK;
    k_vv_second<T><<<dim3((a.max_units + VV_T - 1) / VV_T, a.bt.B), VV_T, 0, st>>>(a, kin_atom);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

__global__ void k_kinetic(int n, const double *__restrict__ v, const double *__restrict__ m, double *__restrict__ kin)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = v[3 * i], b = v[3 * i + 1], c = v[3 * i + 2];
    kin[i] = 0.5 * m[i] * (a * a + b * b + c * c);
}

__global__ void k_inverse(int n, const double *__restrict__ m, double *__restrict__ im)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) im[i] = 1.0 / m[i];
}

int launch_inverse(int n, const double *m, double *im, cudaStream_t st)
{
    if (n <= 0) return MSM_OK;
    k_inverse<<<(n + 255) / 256, 256, 0, st>>>(n, m, im);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

int launch_kinetic(int n, const double *v, const double *m, double *kin_atom, cudaStream_t st)
{
    if (n <= 0) return MSM_OK;
    k_kinetic<<<(n + 255) / 256, 256, 0, st>>>(n, v, m, kin_atom);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// One thread per system: uk[s*uk_stride + 2*step + (0, 1)] = (U_s, K_s), step = *ctr.
__global__ void k_record_uk(int B, const double *__restrict__ sums, int sums_stride, const double *__restrict__ kin,
                            double *__restrict__ uk, int uk_stride, int *__restrict__ ctr, bool add_slow)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int step = *ctr;
    if (s < B) {
        uk[(size_t)s * uk_stride + 2 * step] = add_slow ? sums[s * sums_stride] + sums[s * sums_stride + 2]
                                                        : sums[s * sums_stride];
        uk[(size_t)s * uk_stride + 2 * step + 1] = kin[s];
    }
    __syncthreads();
    if (threadIdx.x == 0 && blockIdx.x == 0 && gridDim.x == 1) *ctr = step + 1;
}

int launch_record_uk(int B, const double *sums, int sums_stride, const double *kin, double *uk, int uk_stride,
                     int *ctr, bool add_slow, cudaStream_t st)
{
    if (B > 1024) return fail_msg(MSM_EINVAL, "at most 1024 systems record energies");
    k_record_uk<<<1, 1024, 0, st>>>(B, sums, sums_stride, kin, uk, uk_stride, ctr, add_slow);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

__global__ void k_add(int64_t n, const double *__restrict__ x, double *__restrict__ y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

int launch_add(int64_t n, const double *x, double *y, cudaStream_t st)
{
    if (n <= 0) return MSM_OK;
    k_add<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x, y);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template int launch_vv_first<float>(const VVArgs &, cudaStream_t);
template int launch_vv_first<double>(const VVArgs &, cudaStream_t);
template int launch_vv_second<float>(const VVArgs &, double *, cudaStream_t);
template int launch_vv_second<double>(const VVArgs &, double *, cudaStream_t);

// --------------------------------------------------------------- parareal

constexpr int PR_T = 256;

__global__ void k_pr_update(int count, const double *__restrict__ f, const double *__restrict__ gnew,
                            const double *__restrict__ gold, double *__restrict__ out,
                            const double *__restrict__ prev, double *__restrict__ part)
{
    __shared__ double ws[PR_T / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double dx = 0;
    if (i < count) {
        const double v = f[i] + (gnew[i] - gold[i]);     // the bracket is exactly 0 when gnew == gold bitwise
        out[i] = v;
        if (prev) dx = fabs(v - prev[i]);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) dx = fmax(dx, __shfl_xor_sync(0xffffffffu, dx, o));
    if (lane == 0) ws[w] = dx;
    __syncthreads();
    if (threadIdx.x == 0 && part) {
        double r = 0;
        for (int k = 0; k < PR_T / 32; k++) r = fmax(r, ws[k]);
        part[blockIdx.x] = r;
    }
}

int launch_parareal_update(int count, const double *f, const double *gnew, const double *gold, double *out,
                           const double *prev, double *dx_partials, cudaStream_t st)
{
    if (count <= 0) return MSM_OK;
    k_pr_update<<<(count + PR_T - 1) / PR_T, PR_T, 0, st>>>(count, f, gnew, gold, out, prev, dx_partials);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Rigid-molecule projection after a parareal correction (the water
// completion's reading; the paper has no constraints): the correction
// F + (G_new - G_old) adds molecules from different trajectories, so a
// molecule whose squared bond lengths miss the rigid ones by more than
// `thresh` (relative) is projected back -- positions by SHAKE iterations along
// its own current bond vectors (inverse-mass weights) until every bond is
// within `tol`, then velocities by the RATTLE velocity stage (|rv| <= tol_v).
// Other molecules are not touched, bit for bit.  FP64, one thread per molecule.
__global__ void k_pr_project(int n_mol, double *__restrict__ x, double *__restrict__ v, const double *__restrict__ m,
                             double d_oh2, double d_hh2, double thresh, double tol, double tol_v, int max_iter,
                             int *__restrict__ status)
{
    const int mo = blockIdx.x * blockDim.x + threadIdx.x;
    if (mo >= n_mol) return;
    const int i0 = 3 * mo;
    const double d2[3] = {d_oh2, d_oh2, d_hh2};
    double p[3][3], w[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        w[a] = 1.0 / m[i0 + a];
#pragma unroll
        for (int d = 0; d < 3; d++) p[a][d] = x[3 * (i0 + a) + d];
    }
    bool off = false;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int a = bond_i(c), b = bond_j(c);
        double r2 = 0;
#pragma unroll
        for (int d = 0; d < 3; d++) { const double t = p[a][d] - p[b][d]; r2 += t * t; }
        if (fabs(d2[c] - r2) > thresh * d2[c]) off = true;
    }
    if (!off) return;
    bool ok = false;
    for (int it = 0; it < max_iter && !ok; it++) {
        ok = true;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int a = bond_i(c), b = bond_j(c);
            double r[3], r2 = 0;
#pragma unroll
            for (int d = 0; d < 3; d++) { r[d] = p[a][d] - p[b][d]; r2 += r[d] * r[d]; }
            const double diff = d2[c] - r2;
            if (fabs(diff) <= tol * d2[c]) continue;
            ok = false;
            const double g = diff / (2.0 * r2 * (w[a] + w[b]));
#pragma unroll
            for (int d = 0; d < 3; d++) { p[a][d] += g * w[a] * r[d]; p[b][d] -= g * w[b] * r[d]; }
        }
    }
    if (!ok) { atomicCAS(status, 0, MSM_ENOCONV); return; }
    double u[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int d = 0; d < 3; d++) u[a][d] = v[3 * (i0 + a) + d];
    ok = false;
    for (int it = 0; it < max_iter && !ok; it++) {
        ok = true;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int a = bond_i(c), b = bond_j(c);
            double r[3], r2 = 0, rv = 0;
#pragma unroll
            for (int d = 0; d < 3; d++) {
                r[d] = p[a][d] - p[b][d];
                r2 += r[d] * r[d];
                rv += r[d] * (u[a][d] - u[b][d]);
            }
            if (fabs(rv) <= tol_v) continue;
            ok = false;
            const double k = rv / (r2 * (w[a] + w[b]));
#pragma unroll
            for (int d = 0; d < 3; d++) { u[a][d] -= k * w[a] * r[d]; u[b][d] += k * w[b] * r[d]; }
        }
    }
    if (!ok) atomicCAS(status, 0, MSM_ENOCONV);
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int d = 0; d < 3; d++) { x[3 * (i0 + a) + d] = p[a][d]; v[3 * (i0 + a) + d] = u[a][d]; }
}

int launch_pr_project(int n_mol, double *x, double *v, const double *m, double d_oh2, double d_hh2, double thresh,
                      double tol, double tol_v, int *status, cudaStream_t st)
{
    if (n_mol <= 0) return MSM_OK;
    k_pr_project<<<(n_mol + 127) / 128, 128, 0, st>>>(n_mol, x, v, m, d_oh2, d_hh2, thresh, tol, tol_v, 1000, status);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Per-block max |a_i - b_i| (the parareal convergence measure).
__global__ void k_absdiff_partials(int count, const double *__restrict__ a, const double *__restrict__ b,
                                   double *__restrict__ part)
{
    __shared__ double ws[PR_T / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double dx = i < count ? fabs(a[i] - b[i]) : 0.0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) dx = fmax(dx, __shfl_xor_sync(0xffffffffu, dx, o));
    if (lane == 0) ws[w] = dx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0;
        for (int k = 0; k < PR_T / 32; k++) r = fmax(r, ws[k]);
        part[blockIdx.x] = r;
    }
}

int launch_absdiff_partials(int count, const double *a, const double *b, double *part, cudaStream_t st)
{
    if (count <= 0) return MSM_OK;
    k_absdiff_partials<<<(count + PR_T - 1) / PR_T, PR_T, 0, st>>>(count, a, b, part);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

__global__ void k_max_reduce(int m, const double *__restrict__ v, double *__restrict__ out)
{
    __shared__ double ws[PR_T / 32];
    double r = 0;
    for (int i = threadIdx.x; i < m; i += PR_T) r = fmax(r, v[i]);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) ws[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < PR_T / 32; k++) t = fmax(t, ws[k]);
        *out = t;
    }
}

int launch_max_reduce(int m, const double *v, double *out, cudaStream_t st)
{
    k_max_reduce<<<1, PR_T, 0, st>>>(m, v, out);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Per-segment maxima: out[s] = max(v[s*m .. s*m + m)), one block per segment.
__global__ void k_max_reduce_seg(int m, const double *__restrict__ v, double *__restrict__ out)
{
    __shared__ double ws[PR_T / 32];
    const double *vs = v + (size_t)blockIdx.x * m;
    double r = 0;
    for (int i = threadIdx.x; i < m; i += PR_T) r = fmax(r, vs[i]);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o; o >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
    if (lane == 0) ws[w] = r;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int k = 0; k < PR_T / 32; k++) t = fmax(t, ws[k]);
        out[blockIdx.x] = t;
    }
}

int launch_max_reduce_seg(int nseg, int m, const double *v, double *out, cudaStream_t st)
{
    if (nseg <= 0) return MSM_OK;
    k_max_reduce_seg<<<nseg, PR_T, 0, st>>>(m, v, out);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// Keep the first failure of a sequence of propagations: src is a propagation's
// status word (reset by its next run), dst[0..3] = (code, kind, tag, atom + 1)
// of the first one that failed, tag = the caller's label of that propagation.
__global__ void k_status_fold(const int *__restrict__ src, int *__restrict__ dst, int tag)
{
    if (src[0] != 0 && dst[0] == 0) {
        dst[0] = src[0]; dst[1] = src[1]; dst[2] = tag; dst[3] = src[3];
    }
}

int launch_status_fold(const int *src, int *dst, int tag, cudaStream_t st)
{
    k_status_fold<<<1, 1, 0, st>>>(src, dst, tag);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ----------------------------------------------------------------- utility

__global__ void k_cast_f64(int m, const double *__restrict__ s, float *__restrict__ d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) d[i] = (float)s[i];
}

int launch_cast_f64(int m, const double *src, float *dst, cudaStream_t st)
{
    if (m <= 0) return MSM_OK;
    k_cast_f64<<<(m + 255) / 256, 256, 0, st>>>(m, src, dst);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

}  // namespace msm
