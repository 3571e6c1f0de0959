// Instantiations of the fine-sweep kernel with a stored velocity perturbation
// (FINE_MODE_IMPLICIT_PERT), both Krylov types (a translation unit of its own so that the
// build compiles them beside the others).
#include "fine_kernel.cuh"

namespace pr {

template <typename KT, int W>
static FineFn pick_pert(int KF, int KS) {
#define PR_FINE_CASE(F, S_) \
    if (KF <= F && KS <= S_) return fine_kernel<KT, W, F, S_, FINE_MODE_IMPLICIT_PERT>;
    PR_FINE_CASE(2, 1)
    PR_FINE_CASE(3, 1)
    PR_FINE_CASE(3, 2)
    PR_FINE_CASE(4, 2)
#undef PR_FINE_CASE
    return nullptr;
}

FineFn fine_fn_pert(bool fp32, int W, int KF, int KS) {
    if (fp32) return W == 4 ? pick_pert<float, 4>(KF, KS) : pick_pert<float, 1>(KF, KS);
    return W == 4 ? pick_pert<double, 4>(KF, KS) : pick_pert<double, 1>(KF, KS);
}

}  // namespace pr
