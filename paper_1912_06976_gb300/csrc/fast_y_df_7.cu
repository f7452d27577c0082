// fast_y_df_7.cu -- double-float (GM_DF64) column-direction kernels for the ladder length(s)
// 768.  The double-float kernels are long straight-line code, so their lengths are spread over
// several translation units that compile in parallel.
#include "gm_fast_impl.cuh"

namespace gm {

namespace {
// the lengths LO..HI of the ladder (a template, so that the other lengths are not instantiated)
template <int LO, int HI>
const YOps<dfr> *pick(int N) {
#define F(n, a, b)                                              \
    if constexpr (n >= LO && n <= HI) {                         \
        if (N == n) {                                           \
            static const YOps<dfr> ops = make_yops<dfr, a, b>();     \
            return &ops;                                        \
        }                                                       \
    }
    GM_Y_LADDER_B(F)
#undef F
    return nullptr;
}
}  // namespace

const YOps<dfr> *y_ops_df_7(int N) { return pick<768, 768>(N); }

}  // namespace gm
