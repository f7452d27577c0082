// fast_x_f32.cu -- FP32 row-direction kernels for every length of the row ladder.
#include "gm_fast_impl.cuh"

namespace gm {

const XOps<float> *x_ops_f32(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const XOps<float> ops = make_xops<float, a, b>();             \
        return &ops;                                             \
    }
    GM_X_LADDER(F)
#undef F
    return nullptr;
}

}  // namespace gm
