// hot_interact.cu -- the fixed-order instantiations of the interaction kernels
// (hot_interact.cuh): forces and the adjoint's sink pass.
#include "hot_interact.cuh"

namespace {

// The kernel of the context's force smoothing.
template <int P, class T, int NS, int MODE>
int launch_interact(hot_ctx *c, cudaStream_t s, int cls, unsigned *work, double *acc, double *pot, const T *wsink,
                    double *gsink)
{
    if (c->prm.softening == HOT_SOFT_K1)
        return launch_interact_s<P, T, NS, MODE, HOT_SOFT_K1>(c, s, cls, work, acc, pot, wsink, gsink);
    if (c->prm.softening == HOT_SOFT_SPLINE)
        return launch_interact_s<P, T, NS, MODE, HOT_SOFT_SPLINE>(c, s, cls, work, acc, pot, wsink, gsink);
    return launch_interact_s<P, T, NS, MODE, HOT_SOFT_PLUMMER>(c, s, cls, work, acc, pot, wsink, gsink);
}

template <int P>
int forces_p(hot_ctx *c, double *acc, double *pot)
{
    unsigned *work = (unsigned *)(c->sizes.p + 56);
    if (c->prm.precision == HOT_FP64)
        return launch_interact<P, double, 1, 0>(c, c->st, 0, work, acc, pot, nullptr, nullptr);
    if constexpr (P >= 5) {
        // large expansions: groups of more than 32 sinks run two sinks per lane, so that
        // every coefficient read from shared memory feeds two independent evaluations.  The
        // two classes run concurrently (the second on the second stream, with its own work
        // counter), so that each fills the other's tail of idle SMs.
        unsigned *work2 = (unsigned *)(c->sizes.p + 57);
        HOT_CK(cudaEventRecord(c->ev_fork, c->st));
        HOT_CK(cudaStreamWaitEvent(c->st2, c->ev_fork, 0));
        int r = launch_interact<P, float, 2, 0>(c, c->st2, 2, work2, acc, pot, nullptr, nullptr);
        const int r1 = launch_interact<P, float, 1, 0>(c, c->st, 1, work, acc, pot, nullptr, nullptr);
        HOT_CK(cudaEventRecord(c->ev_join, c->st2));
        HOT_CK(cudaStreamWaitEvent(c->st, c->ev_join, 0));
        return r ? r : r1;
    }
    return launch_interact<P, float, 1, 0>(c, c->st, 0, work, acc, pot, nullptr, nullptr);
}

}  // namespace

int hot_impl_forces(hot_ctx *c, double *acc, double *pot)
{
    hot_tic(c, 4);
    int r;
    if (c->varq) {
        r = hot_impl_forces_vq(c, acc, pot);
        hot_toc(c, 4);
        return r;
    }
    switch (c->p_mom) {
        case 0: r = forces_p<0>(c, acc, pot); break;
        case 1: r = forces_p<1>(c, acc, pot); break;
        case 2: r = forces_p<2>(c, acc, pot); break;
        case 3: r = forces_p<3>(c, acc, pot); break;
        case 4: r = forces_p<4>(c, acc, pot); break;
        case 5: r = forces_p<5>(c, acc, pot); break;
        case 6: r = forces_p<6>(c, acc, pot); break;
        case 7: r = forces_p<7>(c, acc, pot); break;
        case 8: r = forces_p<8>(c, acc, pot); break;
        default: return HOT_ESTATE;
    }
    // periodic boundaries: the far images' local expansion, added to the tree's forces;
    // background subtraction: the analytic fields of the groups' cube lists and
    // surrounding cubes
    if (!r) r = hot_impl_far_field(c, acc, pot);
    if (!r && c->prm.background) r = hot_impl_bg_box(c, acc, pot);
    hot_toc(c, 4);
    return r;
}

// Sink side of the adjoint: for every sink, d/dx_i of sum over its interactions of
// (u_i . a_i + v_i phi_i), with (u_i, v_i) = wsink[slot] (T4, sorted order); written to
// gsink [N][3] (float64, sorted order).  Launched on stream s.
int hot_impl_adjoint_sink(hot_ctx *c, const void *wsink, double *gsink, cudaStream_t s)
{
    unsigned *work = (unsigned *)(c->sizes.p + 56);
#define HOT_ADJ_SINK(PP)                                                                                 \
    case PP:                                                                                             \
        if (c->prm.precision == HOT_FP64)                                                                \
            return launch_interact<PP, double, 1, 1>(c, s, 0, work, nullptr, nullptr, (const double *)wsink, \
                                                     gsink);                                             \
        return launch_interact<PP, float, 1, 1>(c, s, 0, work, nullptr, nullptr, (const float *)wsink, gsink);
    switch (c->p_mom) {
        HOT_ADJ_SINK(0)
        HOT_ADJ_SINK(1)
        HOT_ADJ_SINK(2)
        HOT_ADJ_SINK(3)
        HOT_ADJ_SINK(4)
        HOT_ADJ_SINK(5)
        HOT_ADJ_SINK(6)
        default: return HOT_ESTATE;
    }
#undef HOT_ADJ_SINK
}
