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
    if (A.vl_ctl && A.vl_ctl[1] == 0 && A.vl_ctl[2] == 0) return;     // the Verlet-list path ran
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
            const int atom = A.perm[slot];
            A.sr[atom] = vec4<T>{-pi.w * ax, -pi.w * ay, -pi.w * az, phi};
            if (MODEL) A.lj[atom] = vec4<T>{lx, ly, lz, le};
        }
    }
}

// ------------------------------------------------------------ FP32, packed
//
// The FP32 path evaluates two j atoms per instruction with Blackwell's packed
// f32x2 arithmetic (sub/mul/fma on register pairs; compares, selects and the
// rsqrt stay scalar).  The warp first finds its candidate rows in parallel
// (one row per lane, compacted by ballot into a shared row list with running
// offsets), then streams the concatenated rows 32 atoms at a time: every chunk
// is full except the last, and a lane finds the row of its atom by binary
// search over the offsets.  Chunks are staged as structure-of-arrays so that
// one 64-bit load broadcasts the x (y, z, q) of two consecutive j atoms.  In the
// water model the LJ sites of a chunk are placed first; the O-O LJ term then
// runs over that prefix only.

typedef unsigned long long f2_t;   // two floats in one 64-bit register pair (lo = first)

__device__ __forceinline__ f2_t f2_pack(float lo, float hi)
{
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2_t v, float &lo, float &hi) { asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v)); }
__device__ __forceinline__ f2_t f2_fma(f2_t a, f2_t b, f2_t c)
{
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2_t f2_mul(f2_t a, f2_t b)
{
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_add(f2_t a, f2_t b)
{
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t f2_sub(f2_t a, f2_t b)
{
    f2_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ float f2_sum(f2_t v) { float a, b; f2_unpack(v, a, b); return a + b; }

constexpr int SR2_MAXROWS = 320;           // candidate rows of one brick (bounded by the cutoff)
constexpr float SR2_FAR = 1.0e6f;          // padding atom: far away, charge 0
constexpr float SR2_EPS = 1.0e-20f;        // keeps rsqrt finite at r = 0 (the i = j pair, charge masked to 0)

struct SR2Smem {
    int rs0[SR_WARPS][SR2_MAXROWS];        // first slot of each candidate row
    int rend[SR_WARPS][SR2_MAXROWS];       // running end offset of each row in the concatenation
    __align__(16) float x[SR_WARPS][32], y[SR_WARPS][32], z[SR_WARPS][32], q[SR_WARPS][32];
    __align__(16) int f[SR_WARPS][32];
};

template <bool MODEL>
__global__ void __launch_bounds__(SR_WARPS * 32) k_short_f32x2(const ShortArgs<float> A)
{
    __shared__ SR2Smem S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int brick = blockIdx.x * SR_WARPS + wid;
    if (brick >= A.nbricks || failed(A.status)) return;
    if (A.vl_ctl && A.vl_ctl[1] == 0 && A.vl_ctl[2] == 0) return;     // the Verlet-list path ran
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
    const float h = (float)A.g.h, inv_h = 1.0f / h;
    const float asel = A.a_sel, asel2 = asel * asel;
    const f2_t a2p = f2_pack(A.a2, A.a2), epsp = f2_pack(SR2_EPS, SR2_EPS);
    const f2_t c0p = f2_pack(A.c0, A.c0), c1p = f2_pack(A.c1, A.c1), c2p = f2_pack(A.c2, A.c2);
    const f2_t d0p = f2_pack(A.d0, A.d0), d1p = f2_pack(A.d1, A.d1);
    const unsigned lt = (1u << lane) - 1u;

    for (int base = 0; base < n_i; base += 32) {
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
        const vec4<float> pi = valid ? A.apos[slot] : vec4<float>{3e18f, 3e18f, 3e18f, 0.f};
        const int fi = (MODEL && valid) ? A.aflag[slot] : -2;
        float lo[3], hi[3];
        lo[0] = warp_min(valid ? pi.x : inf_t<float>()); hi[0] = warp_max(valid ? pi.x : -inf_t<float>());
        lo[1] = warp_min(valid ? pi.y : inf_t<float>()); hi[1] = warp_max(valid ? pi.y : -inf_t<float>());
        lo[2] = warp_min(valid ? pi.z : inf_t<float>()); hi[2] = warp_max(valid ? pi.z : -inf_t<float>());

        // ---- candidate rows, one per lane, compacted into the row list
        const int zlo = max(0, (int)floorf((lo[2] - asel) * inv_h)), zhi = min(nz - 1, (int)floorf((hi[2] + asel) * inv_h));
        const int ylo = max(0, (int)floorf((lo[1] - asel) * inv_h)), yhi = min(ny - 1, (int)floorf((hi[1] + asel) * inv_h));
        const int nyr = yhi - ylo + 1, nr_all = (zhi - zlo + 1) * nyr;
        int nrows = 0, total = 0;
        for (int r0 = 0; r0 < nr_all; r0 += 32) {
            const int r = r0 + lane;
            int s0 = 0, len = 0;
            if (r < nr_all) {
                const int cz = zlo + r / nyr, cy = ylo + r % nyr;
                const float dz = fmaxf(0.f, fmaxf((float)cz * h - hi[2], lo[2] - (float)(cz + 1) * h));
                const float dy = fmaxf(0.f, fmaxf((float)cy * h - hi[1], lo[1] - (float)(cy + 1) * h));
                const float d2 = dy * dy + dz * dz;
                if (d2 < asel2) {
                    const float rx = sqrtf(asel2 - d2);
                    const int xlo = max(0, (int)floorf((lo[0] - rx) * inv_h));
                    const int xhi = min(nx - 1, (int)floorf((hi[0] + rx) * inv_h));
                    if (xlo <= xhi) {
                        const int rb = (cz * ny + cy) * nx;
                        s0 = start[rb + xlo];
                        len = start[rb + xhi + 1] - s0;
                    }
                }
            }
            const unsigned m = __ballot_sync(0xffffffffu, len > 0);
            int incl = len;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) { const int y = __shfl_up_sync(0xffffffffu, incl, o); if (lane >= o) incl += y; }
            const int pos = nrows + __popc(m & lt);
            if (len > 0 && pos < SR2_MAXROWS) { S.rs0[wid][pos] = s0; S.rend[wid][pos] = total + incl; }
            nrows += __popc(m);
            total += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (nrows > SR2_MAXROWS) { set_status(const_cast<int *>(A.status), MSM_EINVAL); return; }
        __syncwarp();

        f2_t phi2 = 0ull, ax2 = 0ull, ay2 = 0ull, az2 = 0ull;
        f2_t lx2 = 0ull, ly2 = 0ull, lz2 = 0ull, le2 = 0ull;
        const f2_t pix = f2_pack(pi.x, pi.x), piy = f2_pack(pi.y, pi.y), piz = f2_pack(pi.z, pi.z);
        const bool any_lj = MODEL && __any_sync(0xffffffffu, fi >= 0 && (fi & 1));
        for (int cb = 0; cb < total; cb += 32) {
            const int cnt = min(32, total - cb);
            // this lane's atom: row by binary search over the running ends
            float jx = SR2_FAR, jy = SR2_FAR, jz = SR2_FAR, jq = 0.f;
            int jf = 0;
            const int want = cb + lane;
            if (lane < cnt) {
                int lo_r = 0, hi_r = nrows - 1;
                while (lo_r < hi_r) {
                    const int mid = (lo_r + hi_r) >> 1;
                    if (S.rend[wid][mid] > want) hi_r = mid; else lo_r = mid + 1;
                }
                const int rstart = lo_r ? S.rend[wid][lo_r - 1] : 0;
                const int js = S.rs0[wid][lo_r] + (want - rstart);
                const vec4<float> p = A.apos[js];
                jx = p.x; jy = p.y; jz = p.z; jq = p.w;
                if (MODEL) jf = A.aflag[js];
            }
            int pos = lane, n_lj = 0;
            if (MODEL) {                                   // LJ sites first, then the rest, then padding
                const bool isl = lane < cnt && (jf & 1);
                const unsigned ml = __ballot_sync(0xffffffffu, isl), mv = __ballot_sync(0xffffffffu, lane < cnt);
                n_lj = __popc(ml);
                pos = isl ? __popc(ml & lt) : (lane < cnt ? n_lj + __popc(mv & ~ml & lt) : lane);
            }
            S.x[wid][pos] = jx; S.y[wid][pos] = jy; S.z[wid][pos] = jz; S.q[wid][pos] = jq;
            if (MODEL) S.f[wid][pos] = lane < cnt ? jf : 0;
            __syncwarp();
#pragma unroll 2
            for (int k = 0; k < cnt; k += 2) {
                const f2_t xj = *reinterpret_cast<const f2_t *>(&S.x[wid][k]);
                const f2_t yj = *reinterpret_cast<const f2_t *>(&S.y[wid][k]);
                const f2_t zj = *reinterpret_cast<const f2_t *>(&S.z[wid][k]);
                const f2_t qj = *reinterpret_cast<const f2_t *>(&S.q[wid][k]);
                const f2_t dx = f2_sub(xj, pix), dy = f2_sub(yj, piy), dz = f2_sub(zj, piz);
                const f2_t r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                float r2a, r2b, qa, qb;
                f2_unpack(r2, r2a, r2b);
                f2_unpack(qj, qa, qb);
                bool ina = (r2a < A.a2) & (r2a > 0.f), inb = (r2b < A.a2) & (r2b > 0.f);
                if (MODEL) {
                    const int2 fj = *reinterpret_cast<const int2 *>(&S.f[wid][k]);
                    ina = ina & (((fi ^ fj.x) >> 1) != 0);
                    inb = inb & (((fi ^ fj.y) >> 1) != 0);
                }
                const f2_t qm = f2_pack(ina ? qa : 0.f, inb ? qb : 0.f);
                const f2_t r2s = f2_add(r2, epsp);
                float sa, sb;
                f2_unpack(r2s, sa, sb);
                const f2_t ri = f2_pack(rsqrtf(sa), rsqrtf(sb));
                const f2_t ri2 = f2_mul(ri, ri);
                const f2_t poly = f2_fma(f2_fma(c2p, r2s, c1p), r2s, c0p);
                phi2 = f2_fma(qm, f2_sub(ri, poly), phi2);
                const f2_t fs = f2_fma(ri2, ri, f2_fma(d1p, r2s, d0p));
                const f2_t sc = f2_mul(qm, fs);
                ax2 = f2_fma(sc, dx, ax2); ay2 = f2_fma(sc, dy, ay2); az2 = f2_fma(sc, dz, az2);
            }
            if (MODEL && any_lj && (fi & 1)) {
                // O-O Lennard-Jones over the chunk's LJ prefix (both flags set, r < a; one O per molecule)
                for (int k = 0; k < n_lj; k += 2) {
                    const f2_t xj = *reinterpret_cast<const f2_t *>(&S.x[wid][k]);
                    const f2_t yj = *reinterpret_cast<const f2_t *>(&S.y[wid][k]);
                    const f2_t zj = *reinterpret_cast<const f2_t *>(&S.z[wid][k]);
                    const int2 fj = *reinterpret_cast<const int2 *>(&S.f[wid][k]);
                    const f2_t dx = f2_sub(xj, pix), dy = f2_sub(yj, piy), dz = f2_sub(zj, piz);
                    const f2_t r2 = f2_fma(dx, dx, f2_fma(dy, dy, f2_mul(dz, dz)));
                    float r2a, r2b;
                    f2_unpack(r2, r2a, r2b);
                    const bool ina = (r2a < A.a2) & (r2a > 0.f) & ((fj.x & 1) != 0) & (((fi ^ fj.x) >> 1) != 0);
                    const bool inb = (r2b < A.a2) & (r2b > 0.f) & ((fj.y & 1) != 0) & (((fi ^ fj.y) >> 1) != 0);
                    const f2_t ri = f2_pack(rsqrtf(ina ? r2a : A.a2), rsqrtf(inb ? r2b : A.a2));
                    const f2_t ir2 = f2_mul(ri, ri), m = f2_pack(ina ? 1.f : 0.f, inb ? 1.f : 0.f);
                    const f2_t sr2 = f2_mul(f2_pack(A.lj_s2, A.lj_s2), ir2);
                    const f2_t sr6 = f2_mul(f2_mul(sr2, sr2), sr2);
                    const f2_t e = f2_fma(f2_pack(A.lj_4eps, A.lj_4eps), f2_fma(sr6, sr6, f2_sub(0ull, sr6)),
                                          f2_pack(-A.lj_shift, -A.lj_shift));
                    le2 = f2_fma(m, e, le2);
                    const f2_t fl = f2_mul(f2_mul(m, f2_pack(A.lj_24eps, A.lj_24eps)),
                                           f2_mul(f2_fma(f2_add(sr6, sr6), sr6, f2_sub(0ull, sr6)), ir2));
                    lx2 = f2_fma(fl, f2_sub(0ull, dx), lx2);
                    ly2 = f2_fma(fl, f2_sub(0ull, dy), ly2);
                    lz2 = f2_fma(fl, f2_sub(0ull, dz), lz2);
                }
            }
            __syncwarp();
        }
        if (valid) {
            const int atom = A.perm[slot];
            A.sr[atom] = vec4<float>{-pi.w * f2_sum(ax2), -pi.w * f2_sum(ay2), -pi.w * f2_sum(az2), f2_sum(phi2)};
            if (MODEL) A.lj[atom] = vec4<float>{f2_sum(lx2), f2_sum(ly2), f2_sum(lz2), f2_sum(le2)};
        }
        __syncwarp();
    }
}

template <typename T>
int launch_short(const ShortArgs<T> &a, bool model, cudaStream_t st)
{
    if (a.nbricks <= 0) return MSM_OK;
    const int grid = (a.nbricks + SR_WARPS - 1) / SR_WARPS;
    // rows per axis of a brick's candidate set: its extent plus 2 a_sel/h, plus rounding slack
    const int pad = (int)ceil(2.0 * (double)a.a_sel / a.g.h) + 3;
    const bool fits = (a.bd[1] + pad) * (a.bd[2] + pad) <= SR2_MAXROWS;
    if (sizeof(T) == sizeof(float) && fits) {
        const ShortArgs<float> &af = reinterpret_cast<const ShortArgs<float> &>(a);
        if (model) k_short_f32x2<true><<<grid, SR_WARPS * 32, 0, st>>>(af);
        else k_short_f32x2<false><<<grid, SR_WARPS * 32, 0, st>>>(af);
    } else {
        if (model) k_short<T, true, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
        else k_short<T, false, false><<<grid, SR_WARPS * 32, 0, st>>>(a);
    }
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
