// k_md.cu -- everything around the MSM evaluation on the MD path:
//   k_exclusions   rigid-water completion: the short-range kernel skipped the
//                  three intramolecular pairs of each (O, H, H) triple, so only
//                  their smooth part k_e q_i q_j gamma(r/a)/a, which the grids
//                  carry, is subtracted here (FP64); together this removes the
//                  full 1/r = g* + gamma(r/a)/a of every excluded pair
//   k_sum_*        deterministic FP64 sums (fixed partition, fixed tree) for
//                  the energy, the virial and the kinetic energy
//   k_vv_first     velocity Verlet (Sec. 2): half kick, drift, then SHAKE
//                  for each rigid triple (one thread per molecule)
//   k_vv_second    second half kick, RATTLE velocity stage, kinetic energy
//   k_pr_update    parareal correction lambda^{k+1}_{n+1} = F + (G_new - G_old)
//                  in FP64 (Sec. 4) with the max |dx| partials
#include "kernels.cuh"

namespace msm {

// ---------------------------------------------------------------- exclusions

__global__ void k_exclusions(const ExclArgs A)
{
    const int mo = blockIdx.x * blockDim.x + threadIdx.x;
    if (mo >= A.n_mol || failed(A.status)) return;
    const int i0 = 3 * mo;
    double x[3][3], q[3], F[3][3] = {{0}}, dphi[3] = {0, 0, 0}, de[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        q[a] = A.q[i0 + a];
#pragma unroll
        for (int d = 0; d < 3; d++) x[a][d] = A.x[3 * (i0 + a) + d];
    }
    const int pi[3] = {0, 0, 1}, pj[3] = {1, 2, 2};
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const int a = pi[c], b = pj[c];
        const double dx = x[a][0] - x[b][0], dy = x[a][1] - x[b][1], dz = x[a][2] - x[b][2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double rho = r / A.a;
        double gam, dgam;                              // gamma(rho), gamma'(rho)
        if (rho < 1.0) {
            const double r2 = rho * rho;
            gam = GAMMA_C0 + GAMMA_C1 * r2 + GAMMA_C2 * r2 * r2;
            dgam = 2.0 * GAMMA_C1 * rho + 4.0 * GAMMA_C2 * r2 * rho;
        } else {
            gam = 1.0 / rho;
            dgam = -1.0 / (rho * rho);
        }
        const double sm = gam / A.a;                   // smooth part of 1/r
        const double e = A.ke * q[a] * q[b] * sm;
        dphi[a] -= A.ke * q[b] * sm;
        dphi[b] -= A.ke * q[a] * sm;
        de[a] -= 0.5 * e;
        de[b] -= 0.5 * e;
        // U_corr = -k_e q_a q_b gamma(r/a)/a  =>  F_a = k_e q_a q_b gamma'(r/a)/a^2 (r_a - r_b)/r
        const double s = A.ke * q[a] * q[b] * dgam / (A.a * A.a * r);
        F[a][0] += s * dx; F[a][1] += s * dy; F[a][2] += s * dz;
        F[b][0] -= s * dx; F[b][1] -= s * dy; F[b][2] -= s * dz;
    }
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int i = i0 + a;
        double v = 0;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            if (A.forces) A.forces[3 * i + d] += F[a][d];
            v += x[a][d] * F[a][d];
        }
        if (A.pot) A.pot[i] += dphi[a];
        A.eatom[i] += de[a];
        A.vatom[i] += v;
    }
}

int launch_exclusions(const ExclArgs &a, cudaStream_t st)
{
    if (a.n_mol <= 0) return MSM_OK;
    k_exclusions<<<(a.n_mol + 127) / 128, 128, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// ---------------------------------------------------------------- FP64 sums

constexpr int SUM_T = 256;
constexpr int SUM_CHUNK = 4096;    // values per block: fixed partition

int sum_partials_needed(int m) { return (m + SUM_CHUNK - 1) / SUM_CHUNK + 1; }

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

__global__ void k_sum_partials(int m, int ncols, SumCols cols, double *__restrict__ part, int nblk,
                               const int *__restrict__ status)
{
    if (status && failed(status)) return;
    const int b0 = blockIdx.x * SUM_CHUNK;
    for (int c = 0; c < ncols; c++) {
        double v = 0;
        for (int i = b0 + threadIdx.x; i < min(m, b0 + SUM_CHUNK); i += SUM_T) v += cols.c[c][i];
        v = block_sum(v);
        if (threadIdx.x == 0) part[c * nblk + blockIdx.x] = v;
    }
}

__global__ void k_sum_final(int nblk, int ncols, const double *__restrict__ part, double *__restrict__ out,
                            const int *__restrict__ status)
{
    if (status && failed(status)) return;
    for (int c = 0; c < ncols; c++) {
        double v = 0;
        for (int i = threadIdx.x; i < nblk; i += SUM_T) v += part[c * nblk + i];
        v = block_sum(v);
        if (threadIdx.x == 0) out[c] = v;
    }
}

int launch_sum(int m, int ncols, const double *const *cols, double *partials, double *out, const int *status,
               cudaStream_t st)
{
    if (ncols > 4) return fail_msg(MSM_EINVAL, "launch_sum: at most 4 columns");
    SumCols sc;
    for (int c = 0; c < 4; c++) sc.c[c] = c < ncols ? cols[c] : nullptr;
    const int nblk = m > 0 ? (m + SUM_CHUNK - 1) / SUM_CHUNK : 1;
    k_sum_partials<<<nblk, SUM_T, 0, st>>>(m, ncols, sc, partials, nblk, status);
    k_sum_final<<<1, SUM_T, 0, st>>>(nblk, ncols, partials, out, status);
    count_launch(2);
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

// --------------------------------------------------------- velocity Verlet

// Units: a molecule (3 atoms, first n_mol units) or a single site.
__device__ __forceinline__ void unit_atoms(int u, int n_mol, int &i0, int &na)
{
    if (u < n_mol) { i0 = 3 * u; na = 3; }
    else { i0 = 3 * n_mol + (u - n_mol); na = 1; }
}

template <typename T>
__global__ void k_vv_first(const VVArgs A)
{
    const int units = A.n_mol + (A.n - 3 * A.n_mol);
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= units || failed(A.status)) return;
    int i0, na;
    unit_atoms(u, A.n_mol, i0, na);
    const double dt = A.dt;
    double xo[3][3], xn[3][3], v[3][3], im[3];
    for (int a = 0; a < na; a++) {
        const int i = i0 + a;
        im[a] = 1.0 / A.m[i];
        for (int d = 0; d < 3; d++) {
            xo[a][d] = A.x[3 * i + d];
            v[a][d] = A.v[3 * i + d] + 0.5 * dt * A.f[3 * i + d] * im[a];     // half kick
            xn[a][d] = xo[a][d] + dt * v[a][d];                               // drift
        }
    }
    if (na == 3) {
        // SHAKE in local coordinates (relative to the old O position), compute type T
        T p[3][3], ro[3][3];
        const int bi[3] = {0, 0, 1}, bj[3] = {1, 2, 2};
        const T d2[3] = {(T)A.d_oh2, (T)A.d_oh2, (T)A.d_hh2};
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) p[a][d] = (T)(xn[a][d] - xo[0][d]);
        for (int c = 0; c < 3; c++)
            for (int d = 0; d < 3; d++) ro[c][d] = (T)(xo[bi[c]][d] - xo[bj[c]][d]);
        T p0[3][3];
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) p0[a][d] = p[a][d];
        bool ok = false;
        for (int it = 0; it < A.max_iter && !ok; it++) {
            ok = true;
            for (int c = 0; c < 3; c++) {
                const int a = bi[c], b = bj[c];
                T rn[3], rn2 = 0, dot = 0;
                for (int d = 0; d < 3; d++) { rn[d] = p[a][d] - p[b][d]; rn2 += rn[d] * rn[d]; }
                const T diff = d2[c] - rn2;
                if (fabs((double)diff) <= A.tol * (double)d2[c]) continue;
                ok = false;
                for (int d = 0; d < 3; d++) dot += ro[c][d] * rn[d];
                const T wa = (T)im[a], wb = (T)im[b];
                const T g = diff / (T(2) * dot * (wa + wb));
                for (int d = 0; d < 3; d++) { p[a][d] += g * wa * ro[c][d]; p[b][d] -= g * wb * ro[c][d]; }
            }
        }
        if (!ok) set_status(A.status, MSM_ENOCONV);
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) {
                const double dp = (double)(p[a][d] - p0[a][d]);
                xn[a][d] = xn[a][d] + dp;
                v[a][d] += dp / dt;
            }
    }
    for (int a = 0; a < na; a++) {
        const int i = i0 + a;
        for (int d = 0; d < 3; d++) {
            A.xo[3 * i + d] = xo[a][d];
            A.x[3 * i + d] = xn[a][d];
            A.v[3 * i + d] = v[a][d];
        }
    }
}

template <typename T>
__global__ void k_vv_second(const VVArgs A, double *__restrict__ kin)
{
    const int units = A.n_mol + (A.n - 3 * A.n_mol);
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= units || failed(A.status)) return;
    int i0, na;
    unit_atoms(u, A.n_mol, i0, na);
    const double dt = A.dt;
    double v[3][3], m[3];
    for (int a = 0; a < na; a++) {
        const int i = i0 + a;
        m[a] = A.m[i];
        for (int d = 0; d < 3; d++) v[a][d] = A.v[3 * i + d] + 0.5 * dt * A.f[3 * i + d] / m[a];
    }
    if (na == 3) {
        // RATTLE velocity stage: zero the bond-parallel relative velocities
        const int bi[3] = {0, 0, 1}, bj[3] = {1, 2, 2};
        T r[3][3], w[3][3], r2[3];
        for (int c = 0; c < 3; c++) {
            r2[c] = 0;
            for (int d = 0; d < 3; d++) {
                r[c][d] = (T)(A.x[3 * (i0 + bi[c]) + d] - A.x[3 * (i0 + bj[c]) + d]);
                r2[c] += r[c][d] * r[c][d];
            }
        }
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) w[a][d] = (T)v[a][d];
        T w0[3][3];
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) w0[a][d] = w[a][d];
        bool ok = false;
        for (int it = 0; it < A.max_iter && !ok; it++) {
            ok = true;
            for (int c = 0; c < 3; c++) {
                const int a = bi[c], b = bj[c];
                T rv = 0;
                for (int d = 0; d < 3; d++) rv += r[c][d] * (w[a][d] - w[b][d]);
                if (fabs((double)rv) <= A.tol_v) continue;
                ok = false;
                const T wa = T(1) / (T)m[a], wb = T(1) / (T)m[b];
                const T k = rv / (r2[c] * (wa + wb));
                for (int d = 0; d < 3; d++) { w[a][d] -= k * wa * r[c][d]; w[b][d] += k * wb * r[c][d]; }
            }
        }
        if (!ok) set_status(A.status, MSM_ENOCONV);
        for (int a = 0; a < 3; a++)
            for (int d = 0; d < 3; d++) v[a][d] += (double)(w[a][d] - w0[a][d]);
    }
    for (int a = 0; a < na; a++) {
        const int i = i0 + a;
        double k2 = 0;
        for (int d = 0; d < 3; d++) { A.v[3 * i + d] = v[a][d]; k2 += v[a][d] * v[a][d]; }
        if (kin) kin[i] = 0.5 * m[a] * k2;
    }
}

template <typename T>
int launch_vv_first(const VVArgs &a, cudaStream_t st)
{
    const int units = a.n_mol + (a.n - 3 * a.n_mol);
    if (units <= 0) return MSM_OK;
    k_vv_first<T><<<(units + 127) / 128, 128, 0, st>>>(a);
    count_launch();
    CUDA_TRY(cudaGetLastError());
    return MSM_OK;
}

template <typename T>
int launch_vv_second(const VVArgs &a, double *kin_atom, cudaStream_t st)
{
    const int units = a.n_mol + (a.n - 3 * a.n_mol);
    if (units <= 0) return MSM_OK;
    k_vv_second<T><<<(units + 127) / 128, 128, 0, st>>>(a, kin_atom);
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

int launch_kinetic(const VVArgs &a, double *kin_atom, cudaStream_t st)
{
    if (a.n <= 0) return MSM_OK;
    k_kinetic<<<(a.n + 255) / 256, 256, 0, st>>>(a.n, a.v, a.m, kin_atom);
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
