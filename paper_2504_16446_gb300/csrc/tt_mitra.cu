// tt_mitra.cu -- SIRT weights and the SIRT-preconditioned gradient descent
// with Nesterov momentum (Section "Standard reconstruction pipelines": SIRT
// as preconditioned weighted least squares, extended to the full model A =
// B_s (x) P_s and accelerated with Nesterov momentum).
//
// Weights from |A| (the SH basis makes A signed; every John-transform
// coefficient is >= 0, so |A| = |B_s| (x) P_s):
//   rho[s,j,k,c] = (sum_i |B_s[c,i]|) (P_s 1)[j,k]       R = W / rho
//   kappa[v,i]   = sum_s (sum_c |B_s[c,i]|) (P_s^T 1)[v]  D = 1 / kappa
// R = 0 on rays whose length in the volume is <= 1e-6 a, D = 0 where
// kappa <= 1e-6 a Y00.  Both sums reuse the projector kernels: P_s 1 is the
// forward projection of a volume whose isotropic channel is 1 (divided by
// B_s[c,0]), sum_s col_s P_s^T 1 is the adjoint of G[s,j,k,i] = col_s[i].
// Iteration t: y = x_t + mu_t (x_t - x_{t-1}), x_{t+1} = y - (eta/2) D grad L_R(y).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>

#include "tt_internal.cuh"

template <typename T>
tt_status tt_grad_enqueue(tt_handle *h, const T *c, const T *I, const T *W, T *g);
tt_status tt_read_loss(tt_handle *h, double *loss_host);
// Early loss (tt_api.cu): loss_publish_begin makes the next adjoint launched
// with reduce_loss publish the loss in the handle's mapped slot and returns
// its sequence number (0 without a slot; the caller clears h->loss_publish
// after enqueuing); read_published_loss waits for it.
unsigned long long loss_publish_begin(tt_handle *h);
tt_status read_published_loss(tt_handle *h, unsigned long long seq, double *loss_host);

using namespace tt;

#define TT_CUDA(call, what)                                          \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::tt::cuda_fail(_e, what);     \
    } while (0)

namespace {

constexpr double kY00 = 0.28209479177387814347;   // 1 / (2 sqrt(pi))

unsigned blocks_for(long long n)
{
    long long b = (n + 255) / 256;
    const long long cap = 32LL * current_sm_count();
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// row_abs[s][c] = sum_i |B[s][c][i]|, col_abs[s][i] = sum_c |B[s][c][i]| (0 for K <= i < KP)
__global__ void k_abs_sums(const double *__restrict__ B, int S, int C, int K, int KP, double *__restrict__ row_abs,
                           double *__restrict__ col_abs)
{
    const long long n = (long long)S * (C + KP);
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / (C + KP)), r = (int)(t % (C + KP));
        const double *Bs = B + (size_t)s * C * K;
        double v = 0.0;
        if (r < C) {
            for (int i = 0; i < K; ++i) v += fabs(Bs[(size_t)r * K + i]);
            row_abs[(size_t)s * C + r] = v;
        } else {
            const int i = r - C;
            if (i < K)
                for (int c = 0; c < C; ++c) v += fabs(Bs[(size_t)c * K + i]);
            col_abs[(size_t)s * KP + i] = v;
        }
    }
}

// Interior of the padded volume (and of its x-innermost copy cpadx, if any):
// channel 0 = 1, the others 0.
template <typename S>
__global__ void k_unit_volume(S *__restrict__ cpad, S *__restrict__ cpadx, int nx, int ny, int nz, int KP)
{
    const long long n = (long long)nx * ny * nz * KP;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / KP;
        const int i = (int)(t - v * KP);
        const int z = (int)(v % nz), y = (int)((v / nz) % ny), x = (int)(v / ((long long)nz * ny));
        const long long o = (((long long)(x + 2) * (ny + 4) + (y + 2)) * (nz + 4) + (z + 2)) * KP + i;
        cpad[o] = S(i == 0 ? 1.0f : 0.0f);
        if (cpadx) cpadx[(((long long)(z + 2) * (ny + 4) + (y + 2)) * (nx + 4) + (x + 2)) * KP + i] = S(i == 0 ? 1.0f : 0.0f);
    }
}

// In place: R holds B_s[c,0] (P_s 1)[j,k]; becomes W / (row_abs (P_s 1)), 0 on missed rays.
template <typename T>
__global__ void k_row_weights(T *__restrict__ R, const T *__restrict__ W, const T *__restrict__ Bp,
                              const double *__restrict__ row_abs, long long n, int npix_s, int C, int CP, int KP,
                              double len_min)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(t % C);
        const int s = (int)(t / ((long long)npix_s * C));
        const double len = (double)R[t] / (double)Bp[((size_t)s * CP + c) * KP];
        const double w = W ? (double)W[t] : 1.0;
        R[t] = len > len_min ? T(w / (row_abs[(size_t)s * C + c] * len)) : T(0);
    }
}

// G[s][j][k][i] = col_abs[s][i]
template <typename S>
__global__ void k_fill_G(S *__restrict__ G, const double *__restrict__ col_abs, long long n, int npix_s, int KP)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const double v = col_abs[(size_t)(t / ((long long)npix_s * KP)) * KP + (int)(t % KP)];
        if constexpr (std::is_same<S, double>::value) G[t] = v;
        else G[t] = S((float)v);
    }
}

template <typename T>
__global__ void k_invert(T *__restrict__ D, long long n, double floor_)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const double k = (double)D[t];
        D[t] = k > floor_ ? T(1.0 / k) : T(0);
    }
}

// x_{t+1} = y - h D g;  y <- x_{t+1} + mu (x_{t+1} - x_t);  x <- x_{t+1}
template <typename T>
__global__ void k_mitra_update(T *__restrict__ x, T *__restrict__ y, const T *__restrict__ g,
                               const T *__restrict__ D, long long n, T half_eta, T mu)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const T xn = y[t] - half_eta * D[t] * g[t];
        const T xo = x[t];
        x[t] = xn;
        y[t] = xn + mu * (xn - xo);
    }
}

template <typename T, typename S>
tt_status sirt_weights_impl(tt_handle *h, const T *W, T *R, T *D)
{
    double *sums = nullptr;
    const size_t n_row = (size_t)h->S * h->C, n_col = (size_t)h->S * h->KP;
    TT_CUDA(cudaMallocAsync((void **)&sums, sizeof(double) * (n_row + n_col), h->stream), "sirt: cudaMallocAsync");
    double *row_abs = sums, *col_abs = sums + n_row;
    const int npix_s = h->nj * h->nk;
    cudaError_t e = cudaSuccess;
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_abs_sums<<<blocks_for((long long)h->S * (h->C + h->KP)), 256, 0, h->stream>>>(h->B64, h->S, h->C, h->K, h->KP,
                                                                                 row_abs, col_abs);
    k_unit_volume<S><<<blocks_for(h->nvox() * h->KP), 256, 0, h->stream>>>(
        (S *)h->cpad, h->xcopy ? (S *)h->cpad + h->pad_vox * h->KP : nullptr, h->N[0], h->N[1], h->N[2], h->KP);
    e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    if (e == cudaSuccess) e = launch_forward<T, S>(h, R, nullptr, nullptr, false);
    if (e == cudaSuccess) {
        prof_begin(h, TT_KSLOT_VECTOR, &ev);
        k_row_weights<T><<<blocks_for(h->ndata()), 256, 0, h->stream>>>(R, W, (const T *)h->Bp, row_abs, h->ndata(),
                                                                      npix_s, h->C, h->CP, h->KP, 1e-6 * h->a);
        k_fill_G<T><<<blocks_for(h->npix() * h->KP), 256, 0, h->stream>>>((T *)h->G, col_abs, h->npix() * h->KP,
                                                                        npix_s, h->KP);
        e = cudaGetLastError();
        prof_end(h, TT_KSLOT_VECTOR, ev);
    }
    if (e == cudaSuccess) e = launch_adjoint<T, S>(h, D);
    if (e == cudaSuccess) {
        prof_begin(h, TT_KSLOT_VECTOR, &ev);
        k_invert<T><<<blocks_for(h->nvox() * h->K), 256, 0, h->stream>>>(D, h->nvox() * h->K, 1e-6 * h->a * kY00);
        e = cudaGetLastError();
        prof_end(h, TT_KSLOT_VECTOR, ev);
    }
    cudaError_t e2 = cudaFreeAsync(sums, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sirt weights");
    if (e2 != cudaSuccess) return cuda_fail(e2, "sirt: cudaFreeAsync");
    return TT_OK;
}

template <typename T>
tt_status sirt_weights(tt_handle *h, const T *W, T *R, T *D)
{
    if constexpr (std::is_same<T, double>::value) {
        return sirt_weights_impl<double, double>(h, W, R, D);
    } else {
        if (h->prec == TT_BF16) return sirt_weights_impl<float, __nv_bfloat16>(h, W, R, D);
        if (h->prec == TT_F16) return sirt_weights_impl<float, __half>(h, W, R, D);
        return sirt_weights_impl<float, float>(h, W, R, D);
    }
}

bool misaligned(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

tt_status check_weights_args(tt_handle *h, bool want_f64, const void *W, const void *R, const void *D)
{
    if (!h) { set_error("tt_sirt_weights: null handle"); return TT_INVALID_ARG; }
    if ((h->prec == TT_F64) != want_f64) {
        set_error("handle precision does not match the entry point (use the _f64 variants with TT_F64)");
        return TT_INVALID_ARG;
    }
    if (!R || !D || misaligned(R) || misaligned(D) || (W && misaligned(W))) {
        set_error("tt_sirt_weights: R and D must be non-null, all pointers 16-byte aligned");
        return TT_INVALID_ARG;
    }
    return TT_OK;
}

}  // namespace

struct tt_mitra {
    tt_handle *h = nullptr;
    long long n = 0;
    void *x = nullptr, *y = nullptr, *g = nullptr, *D = nullptr, *R = nullptr;
    const void *I = nullptr;
    double eta = 1.0, momentum = -1.0;
    int t = 0;
};

static void free_mitra(tt_mitra *m)
{
    if (!m) return;
    cudaFree(m->x); cudaFree(m->y); cudaFree(m->g); cudaFree(m->D); cudaFree(m->R);
    delete m;
}

template <typename T>
static tt_status mitra_step(tt_mitra *m, double *loss_host)
{
    tt_handle *h = m->h;
    // the loss (at y) is read as soon as the adjoint has published it; the
    // update stays in flight behind it
    const unsigned long long seq = loss_host ? loss_publish_begin(h) : 0;
    tt_status s = tt_grad_enqueue<T>(h, (const T *)m->y, (const T *)m->I, (const T *)m->R, (T *)m->g);
    h->loss_publish = 0;
    if (s != TT_OK) return s;
    m->t += 1;
    const double t1 = m->t + 1;   // index of the next extrapolation
    const double mu = m->momentum < 0 ? (t1 - 1.0) / (t1 + 2.0) : m->momentum;
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_mitra_update<T><<<blocks_for(m->n), 256, 0, h->stream>>>((T *)m->x, (T *)m->y, (const T *)m->g,
                                                              (const T *)m->D, m->n, T(0.5 * m->eta), T(mu));
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    if (e != cudaSuccess) return cuda_fail(e, "mitra update");
    if (!loss_host) return TT_OK;
    return seq ? read_published_loss(h, seq, loss_host) : tt_read_loss(h, loss_host);
}

extern "C" {

tt_status tt_sirt_weights(tt_handle *h, const float *W, float *R, float *D)
{
    tt_status s = check_weights_args(h, false, W, R, D);
    return s != TT_OK ? s : sirt_weights<float>(h, W, R, D);
}

tt_status tt_sirt_weights_f64(tt_handle *h, const double *W, double *R, double *D)
{
    tt_status s = check_weights_args(h, true, W, R, D);
    return s != TT_OK ? s : sirt_weights<double>(h, W, R, D);
}

tt_status tt_mitra_create(tt_handle *h, const void *c0, const void *I, const void *W, double eta, double momentum,
                          tt_mitra **out)
{
    if (!out) { set_error("tt_mitra_create: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (!h || !c0 || !I || misaligned(c0) || misaligned(I) || (W && misaligned(W))) {
        set_error("tt_mitra_create: need a handle and 16-byte aligned c0, I (W may be NULL)");
        return TT_INVALID_ARG;
    }
    if (!(eta > 0.0 && eta < 2.0) || !(momentum < 1.0)) {
        set_error("tt_mitra_create: need 0 < eta < 2 and momentum < 1 (negative: Nesterov schedule)");
        return TT_INVALID_ARG;
    }
    tt_mitra *m = new tt_mitra();
    m->h = h;
    m->n = h->nvox() * h->K;
    m->I = I;
    m->eta = eta;
    m->momentum = momentum;
    const size_t vb = h->esize() * m->n, db = h->esize() * h->ndata();
    cudaError_t e = cudaMalloc(&m->x, vb);
    if (e == cudaSuccess) e = cudaMalloc(&m->y, vb);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, vb);
    if (e == cudaSuccess) e = cudaMalloc(&m->D, vb);
    if (e == cudaSuccess) e = cudaMalloc(&m->R, db);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->x, c0, vb, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->y, c0, vb, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) { free_mitra(m); return cuda_fail(e, "tt_mitra_create"); }
    tt_status s = h->prec == TT_F64
                      ? sirt_weights<double>(h, (const double *)W, (double *)m->R, (double *)m->D)
                      : sirt_weights<float>(h, (const float *)W, (float *)m->R, (float *)m->D);
    if (s != TT_OK) { free_mitra(m); return s; }
    *out = m;
    return TT_OK;
}

tt_status tt_mitra_step(tt_mitra *m, double *loss_host)
{
    if (!m) { set_error("tt_mitra_step: null state"); return TT_INVALID_ARG; }
    return m->h->prec == TT_F64 ? mitra_step<double>(m, loss_host) : mitra_step<float>(m, loss_host);
}

tt_status tt_mitra_get(tt_mitra *m, void *c_out, void *R_out, void *D_out, int *iterations)
{
    if (!m) { set_error("tt_mitra_get: null state"); return TT_INVALID_ARG; }
    tt_handle *h = m->h;
    const size_t vb = h->esize() * m->n, db = h->esize() * h->ndata();
    if (c_out) TT_CUDA(cudaMemcpyAsync(c_out, m->x, vb, cudaMemcpyDeviceToDevice, h->stream), "copy x");
    if (R_out) TT_CUDA(cudaMemcpyAsync(R_out, m->R, db, cudaMemcpyDeviceToDevice, h->stream), "copy R");
    if (D_out) TT_CUDA(cudaMemcpyAsync(D_out, m->D, vb, cudaMemcpyDeviceToDevice, h->stream), "copy D");
    if (iterations) *iterations = m->t;
    return TT_OK;
}

tt_status tt_mitra_destroy(tt_mitra *m)
{
    // Does not touch m->h (the handle may already be destroyed); cudaFree
    // waits for the device.
    free_mitra(m);
    return TT_OK;
}

}  // extern "C"
