// Stateless device ops of the C ABI: kernels on caller-owned device arrays.
//
//   lsgg_neighbour_max   Eq. (16)'s max over all other grains and the
//                        ID-field of Sec. 3.1 for a packed set of boxes, through
//                        the per-cell top-2 field (two 64-bit atomicMax of
//                        (value, -index) keys per box cell), in caller scratch.
//   lsgg_neighbour_max_noalloc  the same kernels with the field in a static
//                        device array, for callers that cannot allocate.
#include "lsgg_internal.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

__device__ __forceinline__ bool op_box_ok(const lsgg_box& b, int Nx, int Ny, int Nz, long long n_elems) {
    if (b.nx <= 0) return false;
    if (b.ny < 1 || b.nz < 1 || b.nx > Nx || b.ny > Ny || b.nz > Nz) return false;
    if (b.ox < 0 || b.oy < 0 || b.oz < 0 || b.ox >= Nx || b.oy >= Ny || b.oz >= Nz) return false;
    long long n = (long long)b.nx * b.ny * b.nz;
    return b.offset >= 0 && b.offset + n <= n_elems;
}

__global__ void __launch_bounds__(256)
k_nm_scatter(const lsgg_box* __restrict__ boxes, const float* __restrict__ phip, long long n_elems,
             int Nx, int Ny, int Nz, unsigned long long* __restrict__ T) {
    const int i = blockIdx.x;
    const lsgg_box b = boxes[i];
    if (!op_box_ok(b, Nx, Ny, Nz, n_elems)) return;
    const long long A = (long long)b.nx * b.ny, n = A * b.nz;
    for (long long c = threadIdx.x; c < n; c += blockDim.x) {
        int z = (int)(c / A);
        int rem = (int)(c - z * A);
        int y = rem / b.nx, x = rem - y * b.nx;
        long long g = ((long long)pmod(b.oz + z, Nz) * Ny + pmod(b.oy + y, Ny)) * Nx + pmod(b.ox + x, Nx);
        unsigned long long key = make_key(phip[b.offset + c], i);
        unsigned long long old = atomicMax(&T[2 * g], key);
        if (old) atomicMax(&T[2 * g + 1], old < key ? old : key);
    }
}

__global__ void __launch_bounds__(256)
k_nm_gather(const lsgg_box* __restrict__ boxes, long long n_elems, int Nx, int Ny, int Nz, float eps,
            const unsigned long long* __restrict__ T, float* __restrict__ m, int* __restrict__ id) {
    const int i = blockIdx.x;
    const lsgg_box b = boxes[i];
    if (!op_box_ok(b, Nx, Ny, Nz, n_elems)) return;
    const long long A = (long long)b.nx * b.ny, n = A * b.nz;
    for (long long c = threadIdx.x; c < n; c += blockDim.x) {
        int z = (int)(c / A);
        int rem = (int)(c - z * A);
        int y = rem / b.nx, x = rem - y * b.nx;
        long long g = ((long long)pmod(b.oz + z, Nz) * Ny + pmod(b.oy + y, Ny)) * Nx + pmod(b.ox + x, Nx);
        unsigned long long k1 = T[2 * g], k2 = T[2 * g + 1];
        int id1 = key_id(k1);
        float v;
        int j;
        if (id1 != i) { v = key_val(k1, eps); j = id1; }
        else { v = key_val(k2, eps); j = key_id(k2); }
        if (!(v > -eps)) j = -1;
        m[b.offset + c] = v;
        id[b.offset + c] = j;
    }
}

// Shared by the allocating entry point and any variant that brings its own field.
int neighbour_max_into(const lsgg_box* boxes, int n_boxes, const float* phip, long long n_elems, int nx, int ny,
                       int nz, float eps, unsigned long long* T, float* m, int* id, cudaStream_t s) {
    long long ncell = (long long)nx * ny * nz;
    if (cudaMemsetAsync(T, 0, (size_t)ncell * 16, s) != cudaSuccess) return LSGG_ERR_CUDA;
    k_nm_scatter<<<n_boxes, 256, 0, s>>>(boxes, phip, n_elems, nx, ny, nz, T);
    k_nm_gather<<<n_boxes, 256, 0, s>>>(boxes, n_elems, nx, ny, nz, eps, T, m, id);
    return cudaGetLastError() == cudaSuccess ? LSGG_OK : LSGG_ERR_CUDA;
}

int neighbour_max_check(const lsgg_box* boxes, int n_boxes, const float* phip, long long n_elems, int nx, int ny,
                        int nz, float eps, const float* m, const int* id) {
    if (!boxes || !phip || !m || !id || n_boxes < 0 || n_elems < 0) return LSGG_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 31)) return LSGG_ERR_INVALID_ARG;
    if (!(eps > 0.0f)) return LSGG_ERR_INVALID_ARG;
    return LSGG_OK;
}

}  // namespace lsgg

extern "C" int lsgg_neighbour_max(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phip_dev,
                                  int64_t n_elems, int32_t nx, int32_t ny, int32_t nz, float eps, void* scratch_dev,
                                  float* m_dev, int32_t* id_dev, void* stream) {
    int r = lsgg::neighbour_max_check(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny, nz, eps, m_dev, id_dev);
    if (r != LSGG_OK) return r;
    if (!scratch_dev || (reinterpret_cast<uintptr_t>(scratch_dev) & 15)) return LSGG_ERR_INVALID_ARG;
    if (n_boxes == 0) return LSGG_OK;
    return lsgg::neighbour_max_into(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny, nz, eps,
                                    static_cast<unsigned long long*>(scratch_dev), m_dev, id_dev,
                                    (cudaStream_t)stream);
}

// ---------------------------------------------------------------------------
// no-allocation variant: the top-2 field lives in static device memory
// ---------------------------------------------------------------------------

namespace {

// 2 x u64 per cell: the neighbour-max field of at most LSGG_NOALLOC_MAX_CELLS cells.
static __device__ __align__(256) unsigned long long g_noalloc_field[2 * (size_t)LSGG_NOALLOC_MAX_CELLS];

// Device address of g_noalloc_field in the current device's context.  The
// host-side name is only a stand-in for the device array, so the address is
// looked up on every call: a lookup is not an allocation, and a cached address
// would outlive the context it belongs to (a device reset or a released
// primary context reloads the module, possibly at another address).
int noalloc_field(unsigned long long** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_field);
    if (e != cudaSuccess || !p) { cudaGetLastError(); return LSGG_ERR_CUDA; }
    *out = static_cast<unsigned long long*>(p);
    return LSGG_OK;
}

}  // namespace

extern "C" int lsgg_neighbour_max_noalloc(const lsgg_box* boxes_dev, int32_t n_boxes, const float* phip_dev,
                                          int64_t n_elems, int32_t nx, int32_t ny, int32_t nz, float eps,
                                          float* m_dev, int32_t* id_dev, void* stream) {
    int r = lsgg::neighbour_max_check(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny, nz, eps, m_dev, id_dev);
    if (r != LSGG_OK) return r;
    if ((long long)nx * ny * nz > (long long)LSGG_NOALLOC_MAX_CELLS) return LSGG_ERR_CAPACITY;
    if (n_boxes == 0) return LSGG_OK;
    unsigned long long* field = nullptr;
    if ((r = noalloc_field(&field)) != LSGG_OK) return r;
    return lsgg::neighbour_max_into(boxes_dev, n_boxes, phip_dev, n_elems, nx, ny, nz, eps, field, m_dev, id_dev,
                                    (cudaStream_t)stream);
}
