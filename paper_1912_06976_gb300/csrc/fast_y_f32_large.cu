// fast_y_f32_large.cu -- FP32 column-direction kernels, column ladder above 256.
#include "gm_fast_impl.cuh"

namespace gm {

const YOps<float> *y_ops_f32_large(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const YOps<float> ops = make_yops<float, a, b>();             \
        return &ops;                                             \
    }
    GM_Y_LADDER_B(F)
#undef F
    return nullptr;
}

}  // namespace gm
