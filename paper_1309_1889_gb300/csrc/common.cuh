// common.cuh -- types and small device helpers shared by the kernels of
// libmsm_gb300.so.  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/msm.h"

// Packed 4-vector of the compute type: (x, y, z, w) with natural alignment so
// that one 128-bit (float) or 256-bit (double) access moves a whole atom.
template <typename T> struct alignas(4 * sizeof(T)) vec4 { T x, y, z, w; };

// Smoothing constants of the C^2 Taylor gamma (Sec. 3):
//   gamma(rho) = 15/8 - 5/4 rho^2 + 3/8 rho^4 (rho < 1), 1/rho (rho >= 1).
#define GAMMA_C0 (15.0 / 8.0)
#define GAMMA_C1 (-5.0 / 4.0)
#define GAMMA_C2 (3.0 / 8.0)

// Device status word: the first error wins; every later kernel of the same
// evaluation checks it and returns at once, so no kernel indexes a grid with
// an out-of-box atom.
__device__ __forceinline__ void set_status(int *status, int code) { atomicCAS(status, 0, code); }
__device__ __forceinline__ bool failed(const int *status) { return *(volatile const int *)status != 0; }

// binary64 <-> binary32 conversions on the integer pipe, from the IEEE 754
// bit layouts (sign | exponent | fraction: 1|11|52 and 1|8|23, biases 1023
// and 127).  GB300 issues FP64 instructions, conversions included, at 1/64 of
// the FP32 rate, so kernels that move values between the FP64 state and FP32
// arithmetic convert with integer operations instead.  Results equal the
// hardware conversions (round to nearest, ties to even) wherever the binary32
// value is normal, zero or infinite; NaN stays NaN; magnitudes below the
// binary32 normal range (2^-126) become signed zero in both directions.
__device__ __forceinline__ float f32_of(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7ffu);                  // binary64 biased exponent
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);    // leading 23 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                     // the 29 bits dropped
    unsigned r = ((unsigned)(e - 896) << 23) + m;               // rebias: 1023 - 127 = 896
    // ties to even; a carry out of the fraction steps the exponent (to infinity at the top)
    r += (rest > 0x10000000u) | ((rest == 0x10000000u) & (m & 1u));
    if (e <= 896) r = 0u;
    if (e >= 1151) r = (e == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(r | (hi & 0x80000000u));
}
__device__ __forceinline__ double f64_of(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    unsigned hi = ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3), lo = u << 29;
    if (e == 0u) hi = lo = 0u;
    if (e == 255u) hi |= 0x7ff00000u;
    return __longlong_as_double((long long)(((unsigned long long)(hi | (u & 0x80000000u)) << 32) | lo));
}
// 1/sqrt(x) from the hardware approximation (PTX rsqrt.approx.ftz.f32: relative
// error below 2^-22.9), without the extra instructions the non-FTZ rsqrtf adds
// for subnormal x.  The pair kernels call it only on r^2 + 1e-12, never below
// the normal range.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// T from / to the FP64 state: the integer-pipe conversions for T = float, the
// identity for T = double.
template <typename T> __device__ __forceinline__ T to_t(double x);
template <> __device__ __forceinline__ float to_t<float>(double x) { return f32_of(x); }
template <> __device__ __forceinline__ double to_t<double>(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return f64_of(x); }
__device__ __forceinline__ double to_d(double x) { return x; }

// Geometry of one system's finest-grid cells and grid levels.
struct CellGeom {
    double origin[3];   // box origin x0
    double h;           // finest spacing
    int    nc[3];       // cells per axis: floor(L/h) + 1
    int    ncells;
};

#define MSM_MAX_LEVELS 12

struct LevelGeom {
    int lo[3];          // index of the first point per axis
    int n[3];           // points per axis (x: padded to a multiple of 4, see nx_log)
    int off;            // offset of this level in the concatenated grid buffer
    int nx_log;         // points along x of the method's grid; the n[0] - nx_log points
                        // after them carry zero charge (rows start on 16-byte boundaries)
};

struct GridGeom {
    int       levels;
    LevelGeom L[MSM_MAX_LEVELS];
    int       total;    // points over all levels
};

// One system of a batch.  A batch is B independent systems evaluated by the
// same launches: their atoms, sorted slots, cells and grid points are
// concatenated, and every kernel finds its system's geometry here (the
// system index is blockIdx.y, or the owner of a tile of a persistent
// launch).  A single system is the batch B = 1.  Nothing in a system's
// arithmetic depends on the other systems, so each result equals the
// result of evaluating that system alone, bit for bit.
struct SysDesc {
    CellGeom g;         // finest cells of this system
    GridGeom gg;        // its levels; LevelGeom::off counts from grid_off
    double inv_h;       // 1/h rounded once (the binning contract)
    double box_lo[3], box_hi[3];
    int atom_off, n;    // atoms, and sorted slots, [atom_off, atom_off + n)
    int n_mol;          // leading rigid (O, H, H) triples of the system
    int cell_off;       // global id of its first cell (cell_start index)
    int bd[3], nb[3], nbricks;   // short-range bricks: edge in cells, count per axis
    int lj_bd[3], lj_nb[3], lj_nbricks;   // bricks of the LJ-site pass (water completion)
    int cp_nc[2];       // cluster-pair columns of 2 x 2 cells per axis (x, y)
    int gp_cw, gp_nc[2], gp_col_off;      // i groups of the short-range pass: columns of gp_cw x gp_cw
                                          // cells, count per axis, global index of the first column
    int lgp_cw, lgp_nc[2], lgp_col_off;   // the same for the LJ-site pass
    int col_off;        // global index of its first column
    int zc_off;         // first entry of its columns' layer-prefix tables (nc[2] + 1 per column)
    int grid_off;       // first point of its grids in the concatenated grid buffers
    int top_off;        // first point of its top level in the FP64 top buffer
    int ttab_off;       // first entry of its top-level Toeplitz table
    int part_off;       // first block of its FP64 sum partials
    int wall_lo[3], wall_hi[3];   // only atoms in cells c < wall_lo[d] or c > wall_hi[d] can
                                  // reach the flat-bottom wall (one cell of margin)
};

// 1-D cubic C1 numerical-Hermite weights of an atom whose fractional
// coordinate within its finest cell is f in [0, 1): weights of grid points
// c-1, c, c+1, c+2 (c = the atom's cell), i.e. Phi(f+1), Phi(f), Phi(f-1),
// Phi(f-2), and their derivatives d/df.  Phi(t) = (1-|t|)(1+|t|-3/2 t^2) on
// |t| <= 1 and -1/2 (|t|-1)(2-|t|)^2 on 1 <= |t| <= 2 (Sec. 3, p = 3).
template <typename T>
__device__ __forceinline__ void phi_weights(T f, T w[4])
{
    const T g = T(1) - f;
    w[0] = T(-0.5) * f * g * g;                         // Phi(1 + f)
    w[1] = g * (T(1) + f - T(1.5) * f * f);             // Phi(f)
    w[2] = f * (T(1) + g - T(1.5) * g * g);             // Phi(1 - f)
    w[3] = T(-0.5) * g * f * f;                         // Phi(2 - f)
}

template <typename T>
__device__ __forceinline__ void phi_weights_d(T f, T w[4], T dw[4])
{
    const T g = T(1) - f;
    w[0] = T(-0.5) * f * g * g;
    w[1] = g * (T(1) + f - T(1.5) * f * f);
    w[2] = f * (T(1) + g - T(1.5) * g * g);
    w[3] = T(-0.5) * g * f * f;
    // d/df of each: Phi'(1+f), Phi'(f), -Phi'(1-f), -Phi'(2-f)
    dw[0] = T(-0.5) * g * (T(1) - T(3) * f);            // -1/2 (1-f)(1-3f)
    dw[1] = f * (T(-5) + T(4.5) * f);                   // -5f + 9/2 f^2
    dw[2] = g * (T(5) - T(4.5) * g);                    // 5g - 9/2 g^2, g = 1-f
    dw[3] = T(0.5) * f * (T(3) * f - T(2));             // d/df of -1/2 (1-f) f^2
}

// Kernel launch accounting (reported through msm_kernel_launches()).
void count_launch(int k = 1);

#define CUDA_TRY(expr)                                                    \
    do {                                                                  \
        cudaError_t e__ = (expr);                                         \
        if (e__ != cudaSuccess) return fail_cuda(e__, #expr, __FILE__, __LINE__); \
    } while (0)

int fail_cuda(cudaError_t e, const char *what, const char *file, int line);
int fail_msg(int code, const char *fmt, ...);
