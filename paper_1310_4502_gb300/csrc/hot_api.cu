// hot_api.cu -- the C ABI declared in include/hot.h: context lifetime, argument checks,
// stage ordering, status word, debug copies, hash lookups and the FMA microbenchmark.
#include <cmath>
#include <new>

#include "hot_common.cuh"
#include "generated.cuh"

int hot_impl_lookup(hot_ctx *c, const uint64_t *keys, int64_t n, int32_t *idx);

std::atomic<long long> hot_launch_counter{0};
std::atomic<long long> hot_bytes_held{0}, hot_bytes_peak{0};

namespace {

int status_code(unsigned bits)
{
    if (bits & HOT_ST_INPUT) return HOT_EINPUT;
    if (bits & HOT_ST_TIMEOUT) return HOT_ETIMEOUT;
    if (bits & (HOT_ST_FRONTIER | HOT_ST_HASH)) return HOT_EOVERFLOW;
    if (bits & HOT_ST_INTERNAL) return HOT_ECUDA;
    return HOT_OK;
}

int check_params(const hot_params *p)
{
    if (!p) return HOT_EINVAL;
    if (p->p < 0 || p->p > HOT_PMAX) return HOT_EINVAL;
    if (!(p->tol > 0.0) || !(p->eps >= 0.0) || !(p->G == p->G)) return HOT_EINVAL;
    if (p->leaf_max < 1 || p->group_max < 1 || p->leaf_max > 4096 || p->group_max > (1 << 20)) return HOT_EINVAL;
    if (p->precision != HOT_FP32_MIXED && p->precision != HOT_FP64) return HOT_EINVAL;
    if (p->softening != HOT_SOFT_PLUMMER && p->softening != HOT_SOFT_K1 && p->softening != HOT_SOFT_SPLINE)
        return HOT_EINVAL;
    if (p->p_min < -1 || p->p_min > p->p) return HOT_EINVAL;
    if (!(p->box >= 0.0) || !std::isfinite(p->box) || (p->box > 0.0 && (p->ws < 1 || p->ws > HOT_WS_MAX)))
        return HOT_EINVAL;
    if (p->box > 0.0 && !(std::isfinite(p->box_lo[0]) && std::isfinite(p->box_lo[1]) && std::isfinite(p->box_lo[2])))
        return HOT_EINVAL;
    if (p->box > 0.0 && p->p_min >= 0) return HOT_EINVAL;  // one or the other
    if (p->background != 0 && p->background != 1) return HOT_EINVAL;
    if (p->background &&
        (p->bg_up < 0 || p->bg_up > HOT_MAXLEVEL || p->softening != HOT_SOFT_PLUMMER || p->box > 0.0 ||
         p->p_min >= 0 || p->p > HOT_BG_PMAX))
        return HOT_EINVAL;
    return HOT_OK;
}

// Register-resident FMA chains: 8 independent accumulators per thread.
template <class T>
__global__ void k_fma(T *out, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == (T)-12345.0) out[0] = s;  // keeps the chains alive
}

__global__ void k_axpy(double *__restrict__ y, const double *__restrict__ x, double alpha, int64_t n)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        y[k] += alpha * x[k];
}

}  // namespace

int hot_sync_status(hot_ctx *c)
{
    if (hot_join_moments(c)) return HOT_ECUDA;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return HOT_ECUDA;
    unsigned bits = 0;
    if (cudaMemcpy(&bits, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return HOT_ECUDA;
    if (bits) cudaMemset(c->d_status, 0, sizeof(unsigned));
    return status_code(bits);
}

extern "C" {

int hot_create(hot_ctx **out, const hot_params *prm, void *cuda_stream)
{
    if (!out) return HOT_EINVAL;
    *out = nullptr;
    int e = check_params(prm);
    if (e) return e;
    hot_ctx *c = new (std::nothrow) hot_ctx();
    if (!c) return HOT_ENOMEM;
    c->prm = *prm;
    c->st = (cudaStream_t)cuda_stream;
    if (cudaGetDevice(&c->dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->dev) != cudaSuccess) {
        delete c;
        return HOT_ECUDA;
    }
    if (cudaMalloc((void **)&c->d_status, sizeof(unsigned)) != cudaSuccess) {
        delete c;
        return HOT_ENOMEM;
    }
    cudaMemset(c->d_status, 0, sizeof(unsigned));
    c->h_status = nullptr;
    for (int k = 0; k < ST_TIMING_EVENTS; ++k) cudaEventCreate(&c->ev[k]);
    if (cudaStreamCreateWithFlags(&c->st2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_mfork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_mcomb, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_mjoin, cudaEventDisableTiming) != cudaSuccess) {
        hot_destroy(c);
        return HOT_ECUDA;
    }
    *out = c;
    return HOT_OK;
}

int hot_set_params(hot_ctx *c, const hot_params *prm)
{
    if (!c) return HOT_EINVAL;
    int e = check_params(prm);
    if (e) return e;
    bool rebuild = prm->leaf_max != c->prm.leaf_max || prm->group_max != c->prm.group_max;
    bool remoment = prm->p != c->prm.p || prm->eps != c->prm.eps || prm->G != c->prm.G ||
                    prm->precision != c->prm.precision || prm->softening != c->prm.softening ||
                    prm->p_min != c->prm.p_min || prm->box != c->prm.box || prm->ws != c->prm.ws ||
                    prm->background != c->prm.background;
    c->prm = *prm;
    if (rebuild) c->stage = 0;
    else if (remoment && c->stage > 1) c->stage = 1;
    else if (c->stage > 2) c->stage = 2;
    return HOT_OK;
}

int hot_build_tree(hot_ctx *c, const double *pos, const double *mass, int64_t N)
{
    if (!c || !pos || !mass || N < 1 || N > (int64_t)INT32_MAX / 2) return HOT_EINVAL;
    if (hot_join_moments(c)) return HOT_ECUDA;
    c->stage = 0;
    return hot_impl_build(c, pos, mass, N);
}

int hot_compute_moments(hot_ctx *c, int p)
{
    if (!c || p < 0 || p > HOT_PMAX || c->prm.p_min > p) return HOT_EINVAL;
    if (c->stage < 1) return HOT_ESTATE;
    if (hot_join_moments(c)) return HOT_ECUDA;
    c->prm.p = p;
    c->stage = 1;
    return hot_impl_moments(c, p);
}

int hot_traverse(hot_ctx *c, double tol)
{
    if (!c || !(tol > 0.0)) return HOT_EINVAL;
    if (c->stage < 2) return HOT_ESTATE;
    c->stage = 2;
    c->prm.tol = tol;
    return hot_impl_traverse(c, tol);
}

int hot_evaluate_forces(hot_ctx *c, double *acc, double *pot)
{
    if (!c || !acc) return HOT_EINVAL;
    if (c->stage < 3) return HOT_ESTATE;
    if (hot_join_moments(c)) return HOT_ECUDA;
    return hot_impl_forces(c, acc, pot);
}

int hot_adjoint(hot_ctx *c, const double *g_acc, const double *g_pot, double *g_pos, double *g_mass)
{
    if (!c || !g_acc || !g_pos || !g_mass) return HOT_EINVAL;
    if (c->prm.background) return HOT_EINVAL;  // its frozen-list passes carry no contrast or cube terms
    if (c->stage < 3) return HOT_ESTATE;
    if (hot_join_moments(c)) return HOT_ECUDA;
    return hot_impl_adjoint(c, g_acc, g_pot, g_pos, g_mass);
}

int hot_stage_times(hot_ctx *c, float ms[6])
{
    if (!c || !ms) return HOT_EINVAL;
    if (hot_join_moments(c)) return HOT_ECUDA;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return HOT_ECUDA;
    for (int k = 0; k < 6; ++k) {
        ms[k] = 0.f;
        if (c->ev_used[k]) cudaEventElapsedTime(&ms[k], c->ev[2 * k], c->ev[2 * k + 1]);
    }
    return HOT_OK;
}

int hot_bg_sizes(hot_ctx *c, int64_t out[6])
{
    if (!c || !out) return HOT_EINVAL;
    if (!c->prm.background) return HOT_EINVAL;
    out[0] = c->n_empty;
    out[1] = c->n_box;
    out[2] = c->n_box_eval;
    out[3] = c->n_m2p_con;
    out[4] = c->n_m2p_emp;
    out[5] = c->n_m2p_int - c->n_m2p_con - c->n_m2p_emp;
    return HOT_OK;
}

int hot_sizes(hot_ctx *c, int64_t out[10])
{
    if (!c || !out) return HOT_EINVAL;
    out[0] = c->N;
    out[1] = c->ncell;
    out[2] = c->ngroup;
    out[3] = c->nleaf;
    out[4] = c->maxlevel;
    out[5] = c->n_m2p;
    out[6] = c->n_p2p;
    out[7] = c->n_pairs;
    out[8] = c->n_m2p_int;
    out[9] = hot_launch_counter.load();
    return HOT_OK;
}

int hot_debug_get(hot_ctx *c, int what, void *dst, size_t bytes)
{
    if (c && hot_join_moments(c)) return HOT_ECUDA;
    if (!c || !dst) return HOT_EINVAL;
    const void *src = nullptr;
    size_t need = 0;
    const int64_t N = c->N, nc = c->ncell, ng = c->ngroup;
    const int ncomp = c->p_mom >= 0 ? HOT_NCOMP[c->p_mom] : 0;
    int min_stage = 1;
    switch (what) {
        case HOT_DBG_FRAME: src = c->frame.p; need = 4 * sizeof(double); break;
        case HOT_DBG_SORTED_KEYS: src = c->key.p; need = N * sizeof(uint64_t); break;
        case HOT_DBG_PERM: src = c->idx.p; need = N * sizeof(int32_t); break;
        case HOT_DBG_CELL_KEY: src = c->ckey.p; need = nc * sizeof(uint64_t); break;
        case HOT_DBG_CELL_LEVEL: src = c->clevel.p; need = nc * sizeof(int32_t); break;
        case HOT_DBG_CELL_BEGIN: src = c->cbegin.p; need = nc * sizeof(int32_t); break;
        case HOT_DBG_CELL_COUNT: src = c->ccount.p; need = nc * sizeof(int32_t); break;
        case HOT_DBG_CELL_PARENT: src = c->cparent.p; need = nc * sizeof(int32_t); break;
        case HOT_DBG_CELL_NCHILD: src = c->cnchild.p; need = nc * sizeof(int32_t); break;
        case HOT_DBG_GROUP_CELL: src = c->gcell.p; need = ng * sizeof(int32_t); break;
        case HOT_DBG_GROUP_CENTRE: src = c->gcen.p; need = 3 * ng * sizeof(double); break;
        case HOT_DBG_GROUP_DMAX: src = c->gdmax.p; need = ng * sizeof(double); break;
        case HOT_DBG_CELL_MASS: src = c->cmass.p; need = nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_CELL_COM: src = c->ccom.p; need = 3 * nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_MOMENTS: src = c->cmom.p; need = (size_t)ncomp * nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_CELL_BMAX: src = c->cbmax.p; need = nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_CELL_B1: src = c->cB1.p; need = nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_CELL_B2: src = c->cB2.p; need = nc * sizeof(double); min_stage = 2; break;
        case HOT_DBG_M2P_OFFSETS: src = c->off_m2p.p; need = (ng + 1) * sizeof(int64_t); min_stage = 3; break;
        case HOT_DBG_M2P_CELLS: src = c->l_m2p.p; need = c->n_m2p * sizeof(int32_t); min_stage = 3; break;
        case HOT_DBG_P2P_OFFSETS: src = c->off_p2p.p; need = (ng + 1) * sizeof(int64_t); min_stage = 3; break;
        case HOT_DBG_P2P_CELLS: src = c->l_p2p.p; need = c->n_p2p * sizeof(int32_t); min_stage = 3; break;
        case HOT_DBG_M2P_ORDERS: src = c->l_m2p.p; need = c->n_m2p * sizeof(int32_t); min_stage = 3; break;
        case HOT_DBG_M2P_IMAGES: src = c->l_m2p.p; need = c->n_m2p * sizeof(int32_t); min_stage = 3; break;
        case HOT_DBG_P2P_IMAGES: src = c->l_p2p.p; need = c->n_p2p * sizeof(int32_t); min_stage = 3; break;
        case HOT_DBG_BG_CUBE_OFFSETS:
            src = c->off_box.p; need = (ng + 1) * sizeof(int64_t); min_stage = c->prm.background ? 3 : 99; break;
        case HOT_DBG_BG_CUBES: src = c->l_box.p; need = c->n_box * sizeof(int32_t); min_stage = c->prm.background ? 3 : 99; break;
        case HOT_DBG_BG_GROUP_S: src = c->bg_gS.p; need = ng * sizeof(int32_t); min_stage = c->prm.background ? 3 : 99; break;
        case HOT_DBG_BG_EMPTY_PARENT:
            src = c->bg_eparent.p; need = c->n_empty * sizeof(int32_t); min_stage = c->prm.background ? 2 : 99; break;
        case HOT_DBG_BG_EMPTY_OCTANT:
            src = c->bg_eoct.p; need = c->n_empty * sizeof(int32_t); min_stage = c->prm.background ? 2 : 99; break;
        default: return HOT_EINVAL;
    }
    if (c->stage < min_stage) return HOT_ESTATE;
    if (bytes != need) return HOT_EINVAL;
    if (need == 0) return HOT_OK;
    if (cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, c->st) != cudaSuccess) return HOT_ECUDA;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) return HOT_ECUDA;
    // M2P entries carry their order above HOT_ORDER_SHIFT under order selection; M2P and
    // P2P entries their image above HOT_IMG_SHIFT under periodic boundaries
    const bool per = c->prm.box > 0.0;
    const bool m2p = what == HOT_DBG_M2P_CELLS || what == HOT_DBG_M2P_ORDERS || what == HOT_DBG_M2P_IMAGES;
    const bool p2p = what == HOT_DBG_P2P_CELLS || what == HOT_DBG_P2P_IMAGES;
    if (m2p || p2p) {
        int32_t *e = (int32_t *)dst;
        const int64_t n = m2p ? c->n_m2p : c->n_p2p;
        for (int64_t i = 0; i < n; ++i) {
            const uint32_t v = (uint32_t)e[i];
            if (what == HOT_DBG_M2P_CELLS || what == HOT_DBG_P2P_CELLS)
                e[i] = (int32_t)(per ? (v & HOT_IMG_CELL_MASK) : (c->varq ? (v & HOT_CELL_MASK) : v));
            else if (what == HOT_DBG_M2P_ORDERS)
                e[i] = c->varq ? (int32_t)(v >> HOT_ORDER_SHIFT) : c->p_mom;
            else
                e[i] = per ? (int32_t)(v >> HOT_IMG_SHIFT) : 0;
        }
    }
    return HOT_OK;
}

int hot_lookup(hot_ctx *c, const uint64_t *keys, int64_t n, int32_t *idx)
{
    if (!c || (n > 0 && (!keys || !idx)) || n < 0) return HOT_EINVAL;
    if (c->stage < 1) return HOT_ESTATE;
    if (n == 0) return HOT_OK;
    if (hot_join_moments(c)) return HOT_ECUDA;
    return hot_impl_lookup(c, keys, n, idx);
}

int hot_axpy(hot_ctx *c, double *y, const double *x, double alpha, int64_t n)
{
    if (!c || n < 0 || (n > 0 && (!y || !x))) return HOT_EINVAL;
    if (n == 0) return HOT_OK;
    if (hot_join_moments(c)) return HOT_ECUDA;
    HOT_COUNT_LAUNCH();
    k_axpy<<<hot_blocks(n, 256, c->nsm * 32), 256, 0, c->st>>>(y, x, alpha, n);
    return cudaGetLastError() == cudaSuccess ? HOT_OK : HOT_ECUDA;
}

int hot_fma_peak(hot_ctx *c, int dbl, double *flops)
{
    if (!c || !flops) return HOT_EINVAL;
    if (hot_join_moments(c)) return HOT_ECUDA;
    void *buf = nullptr;
    if (cudaMalloc(&buf, 64) != cudaSuccess) return HOT_ENOMEM;
    const int threads = 256, blocks = c->nsm * 8;
    const int iters = dbl ? 4096 : 65536;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(a, c->st);
        if (dbl)
            k_fma<double><<<blocks, threads, 0, c->st>>>((double *)buf, iters, 0.999999, 1e-7);
        else
            k_fma<float><<<blocks, threads, 0, c->st>>>((float *)buf, iters, 0.999999f, 1e-7f);
        cudaEventRecord(b, c->st);
        if (cudaEventSynchronize(b) != cudaSuccess) {
            cudaFree(buf);
            return HOT_ECUDA;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(buf);
    *flops = 2.0 * 8.0 * (double)iters * threads * blocks / (best * 1e-3);
    return HOT_OK;
}

const char *hot_strerror(int code)
{
    switch (code) {
        case HOT_OK: return "ok";
        case HOT_EINVAL: return "invalid argument";
        case HOT_ESTATE: return "call out of order";
        case HOT_ENOMEM: return "device allocation failed";
        case HOT_EOVERFLOW: return "capacity exceeded";
        case HOT_ECUDA: return "CUDA runtime error";
        case HOT_EINPUT: return "non-finite or non-positive input";
        case HOT_ETIMEOUT: return "bounded device wait expired";
        default: return "unknown error";
    }
}

void hot_destroy(hot_ctx *c)
{
    if (!c) return;
    if (c->st2) cudaStreamSynchronize(c->st2);  // moment work may still be on it
    c->mom_pending = false;
    cudaStreamSynchronize(c->st);
    cudaStream_t s = c->st;
    c->part.release(s); c->frame.release(s); c->key.release(s); c->key2.release(s); c->idx.release(s);
    c->idx2.release(s); c->scan_tmp.release(s); c->spos.release(s);
    c->rs_bhist.release(s); c->rs_goff.release(s); c->rs_ctr.release(s); c->rs_status.release(s);
    c->bg_cen.release(s); c->bg_half.release(s); c->bg_q.release(s); c->bg_mom.release(s); c->bg_rho.release(s);
    c->bg_tab.release(s);
    c->bg_ecnt.release(s); c->bg_eoff.release(s); c->bg_eparent.release(s); c->bg_eoct.release(s);
    c->bg_tc.release(s); c->bg_tcf.release(s); c->cnt_box.release(s); c->off_box.release(s); c->l_box.release(s); c->bg_gS.release(s);
    c->smass.release(s); c->lcp.release(s); c->leaflev.release(s); c->ncell_i.release(s); c->cell_off.release(s);
    c->ckey.release(s); c->clevel.release(s); c->cbegin.release(s); c->ccount.release(s); c->cparent.release(s);
    c->cend.release(s); c->child8.release(s); c->cnchild.release(s); c->level_cells.release(s);
    c->hkey.release(s); c->hval.release(s); c->gflag.release(s); c->goff.release(s); c->gcell.release(s);
    c->gcen.release(s); c->gdmax.release(s); c->sizes.release(s); c->cmass.release(s); c->ccom.release(s);
    c->cmom.release(s); c->cbmax.release(s); c->cB1.release(s); c->cB2.release(s); c->item_off.release(s);
    c->item_cell.release(s); c->item_part.release(s); c->rec32.release(s); c->rec64.release(s); c->prel.release(s);
    c->cnt_m2p.release(s); c->cnt_p2p.release(s); c->off_m2p.release(s); c->off_p2p.release(s);
    c->l_m2p.release(s); c->l_p2p.release(s); c->trav_scratch.release(s);
    c->tcell.release(s); c->tcellf.release(s); c->slot_m2p.release(s); c->slot_p2p.release(s);
    c->gkey.release(s); c->gkey2.release(s); c->gorder.release(s); c->gorder2.release(s);
    c->slice_cnt.release(s); c->slice_off.release(s); c->items.release(s);
    c->cBn.release(s); c->bn_cnt.release(s); c->bn_off.release(s); c->bn_cell.release(s); c->bn_part.release(s);
    c->rcq.release(s);
    c->rcqf.release(s);
    c->per_D.release(s); c->per_part.release(s); c->per_coef.release(s);
    for (int q = 0; q < HOT_ORDERS; ++q) {
        c->rec32q[q].release(s);
        c->rec64q[q].release(s);
    }
    c->adj_w.release(s); c->adj_xhl.release(s); c->adj_gsink.release(s); c->adj_gp2p.release(s);
    c->adj_mbar.release(s); c->tp_key.release(s); c->tp_key2.release(s);
    c->tp_val.release(s); c->tp_val2.release(s); c->tp_start.release(s); c->tp_end.release(s);
    c->it_cnt.release(s); c->it_off.release(s); c->it_cell.release(s); c->it_a.release(s); c->it_b.release(s);
    c->it_part.release(s); c->adj_pp.release(s); c->adj_roff.release(s);
    cudaStreamSynchronize(s);
    if (c->d_status) cudaFree(c->d_status);
    for (int k = 0; k < ST_TIMING_EVENTS; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->st2) {
        cudaStreamSynchronize(c->st2);
        cudaStreamDestroy(c->st2);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_mfork) cudaEventDestroy(c->ev_mfork);
    if (c->ev_mcomb) cudaEventDestroy(c->ev_mcomb);
    if (c->ev_mjoin) cudaEventDestroy(c->ev_mjoin);
    delete c;
}

}  // extern "C"

extern "C" int hot_memory_stats(int64_t out[2], int reset_peak)
{
    if (!out) return HOT_EINVAL;
    out[0] = hot_bytes_held.load();
    out[1] = hot_bytes_peak.load();
    if (reset_peak) hot_bytes_peak.store(out[0]);
    return HOT_OK;
}

extern "C" int hot_synchronize(hot_ctx *c)
{
    if (!c) return HOT_EINVAL;
    return hot_sync_status(c);
}

extern "C" int hot_debug_set(hot_ctx *c, int what, int64_t value)
{
    if (!c) return HOT_EINVAL;
    switch (what) {
        case HOT_DBGSET_FRONTIER_CAP:
            if (value < 1 || value > (1 << 24)) return HOT_EINVAL;
            c->trav_cap = (int)value;
            return HOT_OK;
        case HOT_DBGSET_SLOT_CAP:
            if (value < 1 || value > (1 << 24)) return HOT_EINVAL;
            c->slot_capm = c->slot_capp = value;
            return HOT_OK;
        case HOT_DBGSET_WAIT_POLLS:
            if (value < 0 || value > 0xffffffffll) return HOT_EINVAL;
            c->wait_polls = (uint32_t)value;
            return HOT_OK;
        case HOT_DBGSET_WAIT_PROBE:
            if (value != 0 && value != 1) return HOT_EINVAL;
            c->wait_probe = (int)value;
            return HOT_OK;
        default:
            return HOT_EINVAL;
    }
}
