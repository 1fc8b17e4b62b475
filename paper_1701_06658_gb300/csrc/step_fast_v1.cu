// Tile variant 1 of the register-ring kernels (see step_fast.cuh): per size
// class (box side <= 32, 40, 48) the cells per thread V and the block size.
#include "step_fast.cuh"

namespace lsgg {

FastKernel fast_kernel_v1(int cls, int which) {
    switch (cls) {
        case 0:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 8, 128, 32, 3>,
                                           fast::PredictLayout<32, 5>::bytes, 128}
                              : FastKernel{(const void*)fast::k_correct_fast<8, 128, 32, 2>,
                                           fast::CorrectLayout<32>::bytes, 128};
        case 1:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 8, 224, 40, 1>,
                                           fast::PredictLayout<40, 5>::bytes, 224}
                              : FastKernel{(const void*)fast::k_correct_fast<8, 224, 40, 1>,
                                           fast::CorrectLayout<40>::bytes, 224};
        case 2:
            return which == 0 ? FastKernel{(const void*)fast::k_predict_fast<5, 8, 288, 48, 1>,
                                           fast::PredictLayout<48, 5>::bytes, 288}
                              : FastKernel{(const void*)fast::k_correct_fast<8, 288, 48, 1>,
                                           fast::CorrectLayout<48>::bytes, 288};
        default:
            return FastKernel{nullptr, 0, 0};
    }
}

}  // namespace lsgg
