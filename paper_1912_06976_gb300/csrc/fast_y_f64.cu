// fast_y_f64.cu -- FP64 column-direction kernels, column ladder up to 256.
#include "gm_fast_impl.cuh"

namespace gm {

const YOps<double> *y_ops_f64(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const YOps<double> ops = make_yops<double, a, b>();             \
        return &ops;                                             \
    }
    GM_Y_LADDER_A(F)
#undef F
    return nullptr;
}

}  // namespace gm
