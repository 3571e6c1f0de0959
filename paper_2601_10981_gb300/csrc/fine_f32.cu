// Instantiations of the fine-sweep kernel for the float Krylov type (a translation unit of
// its own so that the build compiles them in parallel).
#include "fine_kernel.cuh"

namespace pr {

template <int W, int MODE>
static FineFn pick(int KF, int KS) {
#define PR_FINE_CASE(F, S_) if (KF <= F && KS <= S_) return fine_kernel<float, W, F, S_, MODE>;
    PR_FINE_CASE(2, 1)
    PR_FINE_CASE(3, 1)
    PR_FINE_CASE(3, 2)
    PR_FINE_CASE(4, 2)
#undef PR_FINE_CASE
    return nullptr;
}

template <int W>
static FineFn pick_mode(int KF, int KS, int mode) {
    switch (mode) {
        case FINE_MODE_IMPLICIT: return pick<W, FINE_MODE_IMPLICIT>(KF, KS);
        case FINE_MODE_IMPLICIT_TD: return pick<W, FINE_MODE_IMPLICIT_TD>(KF, KS);
        case FINE_MODE_RK4: return pick<W, FINE_MODE_RK4>(KF, KS);
        case FINE_MODE_IMPLICIT_PERT: return fine_fn_pert(true, W, KF, KS);
    }
    return nullptr;
}

FineFn fine_fn_f32(int W, int KF, int KS, int mode) {
    return W == 4 ? pick_mode<4>(KF, KS, mode) : pick_mode<1>(KF, KS, mode);
}

}  // namespace pr
