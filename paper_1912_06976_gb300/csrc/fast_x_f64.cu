// fast_x_f64.cu -- FP64 row-direction kernels for every length of the row ladder.
#include "gm_fast_impl.cuh"

namespace gm {

const XOps<double> *x_ops_f64(int N) {
#define F(n, a, b)                                               \
    if (N == n) {                                                 \
        static const XOps<double> ops = make_xops<double, a, b>();             \
        return &ops;                                             \
    }
    GM_X_LADDER(F)
#undef F
    return nullptr;
}

}  // namespace gm
