// msm_noalloc.cu -- msm_cell_list_noalloc: the cell binning and stable sort
// without any device allocation.  Its scratch is a file-scope static device
// array that every GPU loading the library holds until the process exits.
#include <cmath>
#include <mutex>

#include "kernels.cuh"

using namespace msm;

#define MSM_NOALLOC_SCRATCH_BYTES (24u << 20)   // 24 MiB: keys, histogram, scan sums, status word
#define MSM_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_scratch[MSM_NOALLOC_SCRATCH_BYTES];

// Device addresses of g_noalloc_scratch, one per device, looked up on the
// first call made with that device current.  In host code the symbol's name
// is only a stand-in, so kernels receive these addresses instead.
static void *g_scratch_addr[MSM_NOALLOC_MAX_DEVICES];
static std::mutex g_scratch_mu;

static int scratch_address(void **out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MSM_NOALLOC_MAX_DEVICES) return fail_msg(MSM_EINVAL, "device %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail_msg(MSM_ECUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return MSM_OK;
}

// Same binning contract as the evaluation path: t = (x - x0) * (1/h) in IEEE
// FP64, c = floor(t); valid when 0 <= t and c <= floor(L/h) on every axis.
// Writes only the key and the histogram.
__global__ void k_noalloc_keys(int n, const double *__restrict__ pos, CellGeom g, double inv_h, int *__restrict__ key,
                               int *__restrict__ count, int *__restrict__ status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const double x = pos[3 * i + d];
        if (!isfinite(x)) { set_status(status, MSM_EINVAL); key[i] = -1; return; }
        const double t = __dmul_rn(__dsub_rn(x, g.origin[d]), inv_h);
        const double fl = floor(t);
        if (!(t >= 0.0) || fl > (double)(g.nc[d] - 1)) { set_status(status, MSM_ERANGE); key[i] = -1; return; }
        c[d] = (int)fl;
    }
    const int k = (c[2] * g.nc[1] + c[1]) * g.nc[0] + c[0];
    key[i] = k;
    atomicAdd(&count[k], 1);
}

// Device memory of the current device (the one the kernels run on), or
// managed memory.  Host memory and allocations on another GPU are refused:
// the kernels would dereference them on the current device.
static bool device_accessible(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) { cudaGetLastError(); return false; }
    if (at.type == cudaMemoryTypeManaged) return true;
    if (at.type != cudaMemoryTypeDevice) return false;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return false; }
    return at.device == dev;
}

extern "C" int msm_cell_list_noalloc(int64_t n, const double *pos, const double box[6], double h, int32_t *perm,
                                     int32_t *cell_start, int64_t cell_start_len, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    if (n < 0 || !box || !(h > 0) || !std::isfinite(h)) return fail_msg(MSM_EINVAL, "bad n, box or h");
    if (!cell_start || (n > 0 && (!pos || !perm))) return fail_msg(MSM_EINVAL, "pos, perm and cell_start are required");
    CellGeom g;
    int64_t ncells = 1;
    for (int d = 0; d < 3; d++) {
        if (!std::isfinite(box[d]) || !std::isfinite(box[3 + d]) || !(box[3 + d] > 0))
            return fail_msg(MSM_EINVAL, "box must be finite with positive lengths");
        const double nc = floor(box[3 + d] / h) + 1.0;
        if (nc > 4.0e6) return fail_msg(MSM_EINVAL, "box too large for h");
        g.origin[d] = box[d];
        g.nc[d] = (int)nc;
        ncells *= g.nc[d];
    }
    if (ncells > (int64_t)1 << 30) return fail_msg(MSM_EINVAL, "too many cells");
    g.h = h;
    g.ncells = (int)ncells;
    if (cell_start_len < ncells + 1) return fail_msg(MSM_EINVAL, "cell_start needs %lld entries", (long long)(ncells + 1));
    // scratch layout: status[4] | bsum | count[ncells + 1] | key[n], each 256-byte aligned
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_bsum = 256;
    const size_t o_count = o_bsum + up(sizeof(int) * (size_t)scan_scratch_ints((int)ncells));
    const size_t o_key = o_count + up(sizeof(int) * (size_t)(ncells + 1));
    const size_t need = o_key + up(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (need > MSM_NOALLOC_SCRATCH_BYTES)
        return fail_msg(MSM_EINVAL, "msm_cell_list_noalloc: %lld atoms and %lld cells need %zu bytes of scratch, "
                        "more than its fixed %u", (long long)n, (long long)ncells, need, MSM_NOALLOC_SCRATCH_BYTES);
    if ((n > 0 && (!device_accessible(pos) || !device_accessible(perm))) || !device_accessible(cell_start))
        return fail_msg(MSM_EINVAL, "msm_cell_list_noalloc takes device arrays of the current device only");
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    unsigned char *b = static_cast<unsigned char *>(base);
    int *status = reinterpret_cast<int *>(b);
    int *bsum = reinterpret_cast<int *>(b + o_bsum);
    int *count = reinterpret_cast<int *>(b + o_count);
    int *key = reinterpret_cast<int *>(b + o_key);
    // the array keeps the previous call's contents: clear what must start at zero
    CUDA_TRY(cudaMemsetAsync(status, 0, 16, st));
    CUDA_TRY(cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(ncells + 1), st));
    if (n > 0) {
        k_noalloc_keys<<<(int)((n + 255) / 256), 256, 0, st>>>((int)n, pos, g, 1.0 / h, key, count, status);
        count_launch();
        CUDA_TRY(cudaGetLastError());
    }
    rc = launch_sort_by_key((int)n, (int)ncells, key, count, cell_start, perm, bsum, status, st);
    if (rc) return rc;
    int hs = 0;
    CUDA_TRY(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (hs != 0) return fail_msg(hs, hs == MSM_ERANGE ? "an atom lies outside the box" : "non-finite coordinate");
    return MSM_OK;
}
