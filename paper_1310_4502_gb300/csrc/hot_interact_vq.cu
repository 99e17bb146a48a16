// hot_interact_vq.cu -- the interaction kernels with per-interaction order selection
// (hot_interact.cuh with VQ = true): every M2P entry carries its expansion order, records
// of each order are staged with their own length and evaluated by that order's routine.
// Kept in its own translation unit so that it compiles beside the fixed-order kernels.
#include "hot_interact.cuh"

namespace {

template <int P, class T>
int forces_vq_t(hot_ctx *c, double *acc, double *pot)
{
    unsigned *work = (unsigned *)(c->sizes.p + 56);
    if (c->prm.softening == HOT_SOFT_K1)
        return launch_interact_s<P, T, 1, 0, HOT_SOFT_K1, true>(c, c->st, 0, work, acc, pot, nullptr, nullptr);
    if (c->prm.softening == HOT_SOFT_SPLINE)
        return launch_interact_s<P, T, 1, 0, HOT_SOFT_SPLINE, true>(c, c->st, 0, work, acc, pot, nullptr, nullptr);
    return launch_interact_s<P, T, 1, 0, HOT_SOFT_PLUMMER, true>(c, c->st, 0, work, acc, pot, nullptr, nullptr);
}

template <int P>
int forces_vq(hot_ctx *c, double *acc, double *pot)
{
    if (c->prm.precision == HOT_FP64) return forces_vq_t<P, double>(c, acc, pot);
    return forces_vq_t<P, float>(c, acc, pot);
}

}  // namespace

// Forces under per-interaction order selection (orders 1..8 as the largest order; order 0
// alone is never a range).
int hot_impl_forces_vq(hot_ctx *c, double *acc, double *pot)
{
    switch (c->p_mom) {
        case 1: return forces_vq<1>(c, acc, pot);
        case 2: return forces_vq<2>(c, acc, pot);
        case 3: return forces_vq<3>(c, acc, pot);
        case 4: return forces_vq<4>(c, acc, pot);
        case 5: return forces_vq<5>(c, acc, pot);
        case 6: return forces_vq<6>(c, acc, pot);
        case 7: return forces_vq<7>(c, acc, pot);
        case 8: return forces_vq<8>(c, acc, pot);
        default: return HOT_ESTATE;
    }
}
