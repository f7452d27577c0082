// fast_y_f64_large.cu -- FP64 column-direction kernels, column ladder above 256.
#include "gm_fast_impl.cuh"

namespace gm {

const YOps<double> *y_ops_f64_large(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const YOps<double> ops = make_yops<double, a, b>();             \
        return &ops;                                             \
    }
    GM_Y_LADDER_B(F)
#undef F
    return nullptr;
}

}  // namespace gm
