// Tile variant 2 of the register-ring kernels (see step_fast.cuh): per size
// class (box side <= 32, 40, 48) the cells per thread V and the block size.
#include "step_fast.cuh"

namespace lsgg {

FastKernel fast_kernel_v2(int cls, int which) {
    switch (cls) {
        case 0:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 2, 512, 32, 1>,
                                           fast::PredictLayout<32, 5>::bytes, 512}
                              : FastKernel{(const void*)fast::k_correct_fast<2, 512, 32, 1>,
                                           fast::CorrectLayout<32>::bytes, 512};
        case 1:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 10, 160, 40, 1>,
                                           fast::PredictLayout<40, 5>::bytes, 160}
                              : FastKernel{(const void*)fast::k_correct_fast<10, 160, 40, 1>,
                                           fast::CorrectLayout<40>::bytes, 160};
        case 2:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 12, 192, 48, 1>,
                                           fast::PredictLayout<48, 5>::bytes, 192}
                              : FastKernel{(const void*)fast::k_correct_fast<12, 192, 48, 1>,
                                           fast::CorrectLayout<48>::bytes, 192};
        default:
            return FastKernel{nullptr, 0, 0};
    }
}

}  // namespace lsgg
