// fast_x_df_2.cu -- double-float (GM_DF64) row-direction kernels for the ladder length(s)
// 320..560.  The double-float kernels are long straight-line code, so their lengths are spread over
// several translation units that compile in parallel.
#include "gm_fast_impl.cuh"

namespace gm {

namespace {
// the lengths LO..HI of the ladder (a template, so that the other lengths are not instantiated)
template <int LO, int HI>
const XOps<dfr> *pick(int N) {
#define F(n, a, b)                                              \
    if constexpr (n >= LO && n <= HI) {                         \
        if (N == n) {                                           \
            static const XOps<dfr> ops = make_xops<dfr, a, b>();     \
            return &ops;                                        \
        }                                                       \
    }
    GM_X_LADDER(F)
#undef F
    return nullptr;
}
}  // namespace

const XOps<dfr> *x_ops_df_2(int N) { return pick<320, 560>(N); }

}  // namespace gm
