// Host side of the register-ring kernels: variant table, configuration and launch.
#include "lsgg_internal.cuh"
#include "step_fast.cuh"
#include "../../include/lsgg.h"

namespace lsgg {

FastKernel fast_kernel_v0(int cls, int which);
FastKernel fast_kernel_v1(int cls, int which);
FastKernel fast_kernel_v2(int cls, int which);

static FastKernel fast_kernel(int cls, int which, int variant) {
    switch (variant) {
        case 1: return fast_kernel_v1(cls, which);
        case 2: return fast_kernel_v2(cls, which);
        default: return fast_kernel_v0(cls, which);
    }
}

int fast_class_side(int cls) { return cls == 0 ? 32 : cls == 1 ? 40 : cls == 2 ? 48 : 0; }

// Set kernel `which` of class `cls` to tile variant `variant`: attributes, grid, block.
cudaError_t configure_fast_variant(StepBuffers& B, int which, int cls, int variant) {
    FastKernel k = fast_kernel(cls, which, variant);
    if (!k.fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.threads, k.smem);
    if (e != cudaSuccess) return e;
    B.grid[which][cls] = B.n_sm * (occ < 1 ? 1 : occ);
    B.smem[which][cls] = k.smem;
    B.fblock[which][cls] = k.threads;
    B.variant[which][cls] = variant;
    return cudaSuccess;
}

cudaError_t configure_fast(StepBuffers& B, int cls, int n_sm) {
    B.n_sm = n_sm;
    cudaError_t e = configure_fast_variant(B, 0, cls, 0);
    if (e != cudaSuccess) return e;
    return configure_fast_variant(B, 1, cls, 0);
}

cudaError_t launch_fast(const StepBuffers& B, int which, int cls, const Taps& taps, const PhysicsDev& phys,
                        const DebugOut& dbg, cudaStream_t s) {
    FastKernel k = fast_kernel(cls, which, B.variant[which][cls]);
    if (which == 0) {
        void* args[] = {(void*)&B, (void*)&taps, (void*)&phys, (void*)&cls};
        return cudaLaunchKernel(k.fn, dim3(B.grid[0][cls]), dim3(k.threads), args, k.smem, s);
    }
    void* args[] = {(void*)&B, (void*)&phys, (void*)&dbg, (void*)&cls};
    return cudaLaunchKernel(k.fn, dim3(B.grid[1][cls]), dim3(k.threads), args, k.smem, s);
}

// An mbarrier with one expected arrival that never comes: the poll loop must
// give up after `iterations` tries and report it.
__global__ void k_wait_timeout(int iterations, int* out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    bool done = false;
    for (int i = 0; i < iterations && !done; ++i) done = mbar_test(&bar, 0u);
    if (threadIdx.x == 0) *out = done ? 0 : 1;
}

}  // namespace lsgg

extern "C" int lsgg_debug_wait_timeout(int32_t device, int32_t iterations, int32_t* timed_out) {
    if (!timed_out || iterations < 1 || iterations > (1 << 24)) return LSGG_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return LSGG_ERR_CUDA; }
    int* d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return LSGG_ERR_OUT_OF_MEMORY; }
    lsgg::k_wait_timeout<<<1, 32>>>(iterations, d);
    int h = -1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return LSGG_ERR_CUDA;
    *timed_out = h;
    return LSGG_OK;
}
