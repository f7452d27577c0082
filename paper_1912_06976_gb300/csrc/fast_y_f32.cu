// fast_y_f32.cu -- FP32 column-direction kernels, column ladder up to 256.
#include "gm_fast_impl.cuh"

namespace gm {

const YOps<float> *y_ops_f32(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const YOps<float> ops = make_yops<float, a, b>();             \
        return &ops;                                             \
    }
    GM_Y_LADDER_A(F)
#undef F
    return nullptr;
}

}  // namespace gm
