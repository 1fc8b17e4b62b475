// Tile variant 0 of the register-ring kernels (see step_fast.cuh): per size
// class (box side <= 32, 40, 48) the cells per thread V and the block size.
#include "step_fast.cuh"

namespace lsgg {

FastKernel fast_kernel_v0(int cls, int which) {
    switch (cls) {
        case 0:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 4, 256, 32, 2>,
                                           fast::PredictLayout<32, 5>::bytes, 256}
                              : FastKernel{(const void*)fast::k_correct_fast<4, 256, 32, 2>,
                                           fast::CorrectLayout<32>::bytes, 256};
        case 1:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 5, 320, 40, 1>,
                                           fast::PredictLayout<40, 5>::bytes, 320}
                              : FastKernel{(const void*)fast::k_correct_fast<5, 320, 40, 1>,
                                           fast::CorrectLayout<40>::bytes, 320};
        case 2:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 6, 384, 48, 1>,
                                           fast::PredictLayout<48, 5>::bytes, 384}
                              : FastKernel{(const void*)fast::k_correct_fast<6, 384, 48, 1>,
                                           fast::CorrectLayout<48>::bytes, 384};
        default:
            return FastKernel{nullptr, 0, 0};
    }
}

}  // namespace lsgg
