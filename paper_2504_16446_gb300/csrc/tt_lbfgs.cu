// tt_lbfgs.cu -- device-resident L-BFGS (Section "Optimization"): two-loop
// recursion (Nocedal & Wright, Algorithm 7.4, H_0 = gamma I with gamma =
// s.y / y.y of the newest pair), backtracking Armijo line search.  Vectors are
// in the handle's precision; every dot product is accumulated in FP64 and
// the recursion coefficients stay on the device (no host round trip inside
// the two loops).  The host reads back only the loss of each trial point,
// g.d, and the three dot products that decide whether a pair is stored.
#include <cmath>
#include <utility>
#include <vector>

#include "tt_internal.cuh"

template <typename T>
tt_status tt_grad_enqueue(tt_handle *h, const T *c, const T *I, const T *W, T *g);
tt_status tt_read_loss(tt_handle *h, double *loss_host);

using namespace tt;

struct tt_lbfgs {
    tt_handle *h = nullptr;
    int m = 0;
    long long n = 0;
    void *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr, *ss = nullptr, *ys = nullptr;
    std::vector<void *> S, Y;
    std::vector<double> rho, sy, yy;
    int count = 0, head = -1;
    double f = 0.0;
    const void *I = nullptr, *W = nullptr;
    double *scal = nullptr;       // device: alpha[m], coef[m], misc[8]
    double *partials = nullptr;   // device: kDotBlocks
    double *pinned = nullptr;     // host: misc[8]
};

#define TT_CUDA(call, what)                                          \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::tt::cuda_fail(_e, what);     \
    } while (0)

static void free_state(tt_lbfgs *st)
{
    if (!st) return;
    cudaFree(st->x); cudaFree(st->g); cudaFree(st->d); cudaFree(st->xt); cudaFree(st->gt);
    cudaFree(st->ss); cudaFree(st->ys);
    for (void *p : st->S) cudaFree(p);
    for (void *p : st->Y) cudaFree(p);
    cudaFree(st->scal); cudaFree(st->partials);
    if (st->pinned) cudaFreeHost(st->pinned);
    delete st;
}

// misc slots in scal[2m + t]
enum { M_GD = 0, M_GG = 1, M_SY = 2, M_SS = 3, M_YY = 4 };

template <typename T>
static tt_status read_misc(tt_lbfgs *st, int first, int count)
{
    tt_handle *h = st->h;
    TT_CUDA(cudaMemcpyAsync(st->pinned + first, st->scal + 2 * st->m + first, sizeof(double) * count,
                            cudaMemcpyDeviceToHost, h->stream), "lbfgs scalar copy");
    TT_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    return TT_OK;
}

template <typename T>
static tt_status lbfgs_step(tt_lbfgs *st, double *loss_out, int *n_evals_out)
{
    tt_handle *h = st->h;
    const long long n = st->n;
    T *x = (T *)st->x, *g = (T *)st->g, *d = (T *)st->d;
    double *alpha = st->scal, *coef = st->scal + st->m, *misc = st->scal + 2 * st->m;
    double step0 = 1.0;
    bool steepest = st->count == 0;
    if (!steepest) {
        // d = g; first loop newest -> oldest
        TT_CUDA(vec_axpby<T>(h, d, g, n, 1.0, nullptr, 0.0), "lbfgs copy");
        for (int t = 0; t < st->count; ++t) {
            const int i = (st->head - t + st->m) % st->m;
            TT_CUDA(vec_dot<T>(h, (const T *)st->S[i], d, n, st->partials, alpha + i, nullptr, st->rho[i]), "dot");
            TT_CUDA(vec_axpby<T>(h, d, (const T *)st->Y[i], n, -1.0, alpha + i, 1.0), "axpy");
        }
        const double gamma = st->sy[st->head] / st->yy[st->head];
        TT_CUDA(vec_axpby<T>(h, d, d, n, 0.0, nullptr, gamma), "scale");
        for (int t = st->count - 1; t >= 0; --t) {
            const int i = (st->head - t + st->m) % st->m;
            TT_CUDA(vec_dot<T>(h, (const T *)st->Y[i], d, n, st->partials, coef + i, alpha + i, -st->rho[i]), "dot");
            TT_CUDA(vec_axpby<T>(h, d, (const T *)st->S[i], n, 1.0, coef + i, 1.0), "axpy");
        }
        TT_CUDA(vec_axpby<T>(h, d, d, n, 0.0, nullptr, -1.0), "negate");
        TT_CUDA(vec_dot<T>(h, g, d, n, st->partials, misc + M_GD, nullptr, 1.0), "dot");
        tt_status s = read_misc<T>(st, M_GD, 1);
        if (s != TT_OK) return s;
        if (!(st->pinned[M_GD] < 0.0)) steepest = true;   // not a descent direction: clear the memory
    }
    double gd;
    if (steepest) {
        st->count = 0;
        st->head = -1;
        TT_CUDA(vec_axpby<T>(h, d, g, n, -1.0, nullptr, 0.0), "lbfgs -g");
        TT_CUDA(vec_dot<T>(h, g, g, n, st->partials, misc + M_GG, nullptr, 1.0), "dot");
        tt_status s = read_misc<T>(st, M_GG, 1);
        if (s != TT_OK) return s;
        const double gg = st->pinned[M_GG];
        if (!(gg > 0.0) || !std::isfinite(gg)) {
            // stationary point (or non-finite gradient): nothing to do
            if (loss_out) *loss_out = st->f;
            if (n_evals_out) *n_evals_out = 0;
            if (!std::isfinite(gg)) { set_error("gradient is not finite"); return TT_NONFINITE; }
            return TT_OK;
        }
        step0 = 1.0 / std::sqrt(gg);
        gd = -gg;
    } else {
        gd = st->pinned[M_GD];
    }

    const double c1 = 1e-4;
    const int max_evals = 20;
    double a = step0;
    T *xt = (T *)st->xt, *gt = (T *)st->gt;
    for (int ne = 1; ne <= max_evals; ++ne) {
        TT_CUDA(cudaMemcpyAsync(xt, x, sizeof(T) * n, cudaMemcpyDeviceToDevice, h->stream), "copy x");
        TT_CUDA(vec_axpby<T>(h, xt, d, n, a, nullptr, 1.0), "trial point");
        tt_status s = tt_grad_enqueue<T>(h, xt, (const T *)st->I, (const T *)st->W, gt);
        if (s != TT_OK) return s;
        double ft = 0.0;
        s = tt_read_loss(h, &ft);
        if (s != TT_OK && s != TT_NONFINITE) return s;
        if (s == TT_OK && ft <= st->f + c1 * a * gd) {
            // s = xt - x, y = gt - g into scratch; keep the pair only if curvature holds
            T *sv = (T *)st->ss, *yv = (T *)st->ys;
            TT_CUDA(vec_sub<T>(h, sv, xt, x, n), "s");
            TT_CUDA(vec_sub<T>(h, yv, gt, g, n), "y");
            TT_CUDA(vec_dot<T>(h, sv, yv, n, st->partials, misc + M_SY, nullptr, 1.0), "dot");
            TT_CUDA(vec_dot<T>(h, sv, sv, n, st->partials, misc + M_SS, nullptr, 1.0), "dot");
            TT_CUDA(vec_dot<T>(h, yv, yv, n, st->partials, misc + M_YY, nullptr, 1.0), "dot");
            s = read_misc<T>(st, M_SY, 3);
            if (s != TT_OK) return s;
            const double sy = st->pinned[M_SY], ss = st->pinned[M_SS], yy = st->pinned[M_YY];
            if (sy > 1e-10 * std::sqrt(ss) * std::sqrt(yy)) {
                const int slot = (st->head + 1) % st->m;
                std::swap(st->S[slot], st->ss);
                std::swap(st->Y[slot], st->ys);
                st->rho[slot] = 1.0 / sy;
                st->sy[slot] = sy;
                st->yy[slot] = yy;
                st->head = slot;
                if (st->count < st->m) ++st->count;
            }
            std::swap(st->x, st->xt);
            std::swap(st->g, st->gt);
            st->f = ft;
            if (loss_out) *loss_out = ft;
            if (n_evals_out) *n_evals_out = ne;
            return TT_OK;
        }
        a *= 0.5;
    }
    if (loss_out) *loss_out = st->f;
    if (n_evals_out) *n_evals_out = max_evals;
    set_error("line search: no Armijo point within 20 evaluations");
    return TT_LINESEARCH_FAILED;
}

extern "C" {

tt_status tt_lbfgs_create(tt_handle *h, int m, const void *c0, const void *I, const void *W, tt_lbfgs **out)
{
    if (!out) { set_error("tt_lbfgs_create: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (!h || !c0 || !I || m < 1 || m > 64) {
        set_error("tt_lbfgs_create: need a handle, c0, I and 1 <= m <= 64");
        return TT_INVALID_ARG;
    }
    tt_lbfgs *st = new tt_lbfgs();
    st->h = h;
    st->m = m;
    st->n = h->nvox() * h->K;
    st->I = I;
    st->W = W;
    const size_t bytes = h->esize() * st->n;
    void **bufs[] = {&st->x, &st->g, &st->d, &st->xt, &st->gt, &st->ss, &st->ys};
    for (void **b : bufs) {
        cudaError_t e = cudaMalloc(b, bytes);
        if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_create: cudaMalloc"); }
    }
    st->S.assign(m, nullptr);
    st->Y.assign(m, nullptr);
    for (int i = 0; i < m; ++i) {
        cudaError_t e = cudaMalloc(&st->S[i], bytes);
        if (e == cudaSuccess) e = cudaMalloc(&st->Y[i], bytes);
        if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_create: cudaMalloc"); }
    }
    st->rho.assign(m, 0.0);
    st->sy.assign(m, 0.0);
    st->yy.assign(m, 0.0);
    cudaError_t e = cudaMalloc(&st->scal, sizeof(double) * (2 * m + 8));
    if (e == cudaSuccess) e = cudaMalloc(&st->partials, sizeof(double) * kDotBlocks);
    if (e == cudaSuccess) e = cudaMallocHost(&st->pinned, sizeof(double) * 8);
    if (e == cudaSuccess) e = cudaMemcpyAsync(st->x, c0, bytes, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_create"); }
    tt_status s = (h->prec != TT_F64)
                      ? tt_grad_enqueue<float>(h, (const float *)st->x, (const float *)I, (const float *)W, (float *)st->g)
                      : tt_grad_enqueue<double>(h, (const double *)st->x, (const double *)I, (const double *)W,
                                                (double *)st->g);
    if (s == TT_OK) s = tt_read_loss(h, &st->f);
    if (s != TT_OK) { free_state(st); return s; }
    *out = st;
    return TT_OK;
}

tt_status tt_lbfgs_step(tt_handle *h, tt_lbfgs *st, void *c_out, double *loss_host, int *n_evals_host)
{
    if (!h || !st || st->h != h) { set_error("tt_lbfgs_step: state does not belong to this handle"); return TT_INVALID_ARG; }
    tt_status s = (h->prec != TT_F64) ? lbfgs_step<float>(st, loss_host, n_evals_host)
                                      : lbfgs_step<double>(st, loss_host, n_evals_host);
    if (c_out && (s == TT_OK || s == TT_LINESEARCH_FAILED)) {
        cudaError_t e = cudaMemcpyAsync(c_out, st->x, h->esize() * st->n, cudaMemcpyDeviceToDevice, h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "tt_lbfgs_step: copy iterate");
    }
    return s;
}

tt_status tt_lbfgs_get(tt_handle *h, tt_lbfgs *st, void *c_dev, void *g_dev, double *loss_host)
{
    if (!h || !st || st->h != h) { set_error("tt_lbfgs_get: state does not belong to this handle"); return TT_INVALID_ARG; }
    const size_t bytes = h->esize() * st->n;
    if (c_dev) TT_CUDA(cudaMemcpyAsync(c_dev, st->x, bytes, cudaMemcpyDeviceToDevice, h->stream), "copy x");
    if (g_dev) TT_CUDA(cudaMemcpyAsync(g_dev, st->g, bytes, cudaMemcpyDeviceToDevice, h->stream), "copy g");
    if (loss_host) *loss_host = st->f;
    return TT_OK;
}

tt_status tt_lbfgs_destroy(tt_lbfgs *st)
{
    // Does not touch st->h: the handle may already be destroyed.  cudaFree
    // waits for the device, so no pending work of the state is cut short.
    free_state(st);
    return TT_OK;
}

}  // extern "C"
