// fast_df.cu -- lookup of the double-float (GM_DF64) kernel tables over the translation units
// that hold them (fast_x_df_*.cu, fast_y_df_*.cu).
#include "gm_fast_ops.h"

namespace gm {

const XOps<dfr> *x_ops_df_0(int N);
const XOps<dfr> *x_ops_df_1(int N);
const XOps<dfr> *x_ops_df_2(int N);
const XOps<dfr> *x_ops_df_3(int N);
const XOps<dfr> *x_ops_df_4(int N);
const YOps<dfr> *y_ops_df_0(int N);
const YOps<dfr> *y_ops_df_1(int N);
const YOps<dfr> *y_ops_df_2(int N);
const YOps<dfr> *y_ops_df_3(int N);
const YOps<dfr> *y_ops_df_4(int N);
const YOps<dfr> *y_ops_df_5(int N);
const YOps<dfr> *y_ops_df_6(int N);
const YOps<dfr> *y_ops_df_7(int N);

const XOps<dfr> *x_ops_df(int N) {
    const XOps<dfr> *o = nullptr;
    if (!o) o = x_ops_df_0(N);
    if (!o) o = x_ops_df_1(N);
    if (!o) o = x_ops_df_2(N);
    if (!o) o = x_ops_df_3(N);
    if (!o) o = x_ops_df_4(N);
    return o;
}

const YOps<dfr> *y_ops_df(int N) {
    const YOps<dfr> *o = nullptr;
    if (!o) o = y_ops_df_0(N);
    if (!o) o = y_ops_df_1(N);
    if (!o) o = y_ops_df_2(N);
    if (!o) o = y_ops_df_3(N);
    if (!o) o = y_ops_df_4(N);
    if (!o) o = y_ops_df_5(N);
    if (!o) o = y_ops_df_6(N);
    if (!o) o = y_ops_df_7(N);
    return o;
}

}  // namespace gm
