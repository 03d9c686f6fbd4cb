// tt_reg.cu -- regularisers of the loss (Section "Optimization": L2Norm and
// TotalVariation, the Huber norm of the spatial gradient of every basis mode)
// on a volume c [nx][ny][nz][K], with FP64 value reduction.
#include <cmath>

#include "tt_kernels.cuh"

namespace tt {

// value = sum c^2, grad = 2 c.  Grid-stride; per-block FP64 partials.
template <typename T>
__global__ void k_l2(const T *__restrict__ c, long long n, T *__restrict__ grad, double *__restrict__ partials)
{
    __shared__ double red[32];
    double v = 0.0;
    Dot2 a = {0.f, 0.f};           // float: compensated FP32 per thread and across the CTA
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const T x = c[t];
        if constexpr (std::is_same<T, float>::value) dot2_add(a, x, x);
        else v = fma(x, x, v);
        if (grad) grad[t] = T(2) * x;
    }
    if constexpr (std::is_same<T, float>::value) v = dot2_block_sum(a, reinterpret_cast<Dot2 *>(red));
    else v = block_sum(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// Huber total variation of every channel i:
//   g_i(x)_d = c_i(x + e_d) - c_i(x) if x_d + 1 < N_d else 0,  t = |g_i(x)|,
//   value = sum H(t), H(t) = t^2/(2 delta) (t <= delta) or t - delta/2,
//   grad_i(y) = sum_{d: y_d >= 1} w(y - e_d) g_i(y - e_d)_d - w(y) sum_d g_i(y)_d,
//   w = H'(t)/t = 1/delta (t <= delta) or 1/t.
// One thread per (voxel, channel); neighbours come through L1.
template <typename T>
__device__ __forceinline__ void tv_point(const T *__restrict__ c, int x, int y, int z, int nx, int ny, int nz,
                                         int K, int i, T inv_delta, T delta, T (&g)[3], T &w, T &H)
{
    const long long sx = (long long)ny * nz * K, sy = (long long)nz * K, sz = K;
    const T *p = c + (((long long)x * ny + y) * nz + z) * K + i;
    const T c0 = __ldg(p);
    g[0] = (x + 1 < nx) ? __ldg(p + sx) - c0 : T(0);
    g[1] = (y + 1 < ny) ? __ldg(p + sy) - c0 : T(0);
    g[2] = (z + 1 < nz) ? __ldg(p + sz) - c0 : T(0);
    const T t = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    if (t <= delta) {
        w = inv_delta;
        H = T(0.5) * t * t * inv_delta;
    } else {
        w = T(1) / t;
        H = t - T(0.5) * delta;
    }
}

template <typename T>
__global__ void k_tv_huber(const T *__restrict__ c, int nx, int ny, int nz, int K, T delta, T *__restrict__ grad,
                           double *__restrict__ partials)
{
    __shared__ double red[32];
    const long long n = (long long)nx * ny * nz * K;
    const T inv_delta = T(1) / delta;
    double v = 0.0;
    Dot2 a = {0.f, 0.f};           // float: compensated FP32 sum of H
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % K);
        const long long vox = t / K;
        const int z = (int)(vox % nz), y = (int)((vox / nz) % ny), x = (int)(vox / ((long long)nz * ny));
        T g[3], w, H;
        tv_point<T>(c, x, y, z, nx, ny, nz, K, i, inv_delta, delta, g, w, H);
        if constexpr (std::is_same<T, float>::value) dot2_add1(a, H);
        else v += H;
        if (grad) {
            T gr = -w * (g[0] + g[1] + g[2]);
            T gm[3], wm, Hm;
            if (x >= 1) { tv_point<T>(c, x - 1, y, z, nx, ny, nz, K, i, inv_delta, delta, gm, wm, Hm); gr += wm * gm[0]; }
            if (y >= 1) { tv_point<T>(c, x, y - 1, z, nx, ny, nz, K, i, inv_delta, delta, gm, wm, Hm); gr += wm * gm[1]; }
            if (z >= 1) { tv_point<T>(c, x, y, z - 1, nx, ny, nz, K, i, inv_delta, delta, gm, wm, Hm); gr += wm * gm[2]; }
            grad[t] = gr;
        }
    }
    if constexpr (std::is_same<T, float>::value) v = dot2_block_sum(a, reinterpret_cast<Dot2 *>(red));
    else v = block_sum(v, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

static unsigned reg_grid(const tt_handle *h, long long n)
{
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > dot_blocks(h) ? dot_blocks(h) : b));
}

template <typename T>
static tt_status reg_finish(tt_handle *h, unsigned blocks, double *value_host)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "regulariser launch");
    e = launch_reduce(h, h->red, blocks, h->loss_dev + 1, nullptr, 1.0);
    if (e != cudaSuccess) return cuda_fail(e, "regulariser reduce");
    e = cudaMemcpyAsync(h->loss_pinned + 1, h->loss_dev + 1, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "regulariser value copy");
    *value_host = h->loss_pinned[1];
    if (!std::isfinite(*value_host)) {
        set_error("regulariser value is not finite");
        return TT_NONFINITE;
    }
    return TT_OK;
}

template <typename T>
static tt_status l2_impl(tt_handle *h, const T *c, T *grad, double *value_host)
{
    const long long n = h->nvox() * h->K;
    const unsigned blocks = reg_grid(h, n);
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_l2<T><<<blocks, 256, 0, h->stream>>>(c, n, grad, h->red);
    prof_end(h, TT_KSLOT_VECTOR, ev);
    return reg_finish<T>(h, blocks, value_host);
}

template <typename T>
static tt_status tv_impl(tt_handle *h, const T *c, double delta, T *grad, double *value_host)
{
    const long long n = h->nvox() * h->K;
    const unsigned blocks = reg_grid(h, n);
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_tv_huber<T><<<blocks, 256, 0, h->stream>>>(c, h->N[0], h->N[1], h->N[2], h->K, (T)delta, grad, h->red);
    prof_end(h, TT_KSLOT_VECTOR, ev);
    return reg_finish<T>(h, blocks, value_host);
}

static tt_status reg_check(const tt_handle *h, tt_precision want, const void *c, const void *grad, const double *value)
{
    if (!h) { set_error("null handle"); return TT_INVALID_ARG; }
    if ((h->prec == TT_F64) != (want == TT_F64)) {
        set_error("handle precision does not match the entry point");
        return TT_INVALID_ARG;
    }
    if (!c || !value || (reinterpret_cast<uintptr_t>(c) & 15u) || (grad && (reinterpret_cast<uintptr_t>(grad) & 15u))) {
        set_error("regulariser: c and value must be non-null, device pointers 16-byte aligned");
        return TT_INVALID_ARG;
    }
    return TT_OK;
}

}  // namespace tt

using namespace tt;

extern "C" {

tt_status tt_l2_norm(tt_handle *h, const float *c, float *grad, double *value_host)
{
    tt_status st = reg_check(h, TT_F32, c, grad, value_host);
    return st != TT_OK ? st : l2_impl<float>(h, c, grad, value_host);
}

tt_status tt_l2_norm_f64(tt_handle *h, const double *c, double *grad, double *value_host)
{
    tt_status st = reg_check(h, TT_F64, c, grad, value_host);
    return st != TT_OK ? st : l2_impl<double>(h, c, grad, value_host);
}

tt_status tt_tv_huber(tt_handle *h, const float *c, double delta, float *grad, double *value_host)
{
    tt_status st = reg_check(h, TT_F32, c, grad, value_host);
    if (st == TT_OK && !(delta > 0.0 && std::isfinite(delta))) { set_error("delta must be positive"); st = TT_INVALID_ARG; }
    return st != TT_OK ? st : tv_impl<float>(h, c, delta, grad, value_host);
}

tt_status tt_tv_huber_f64(tt_handle *h, const double *c, double delta, double *grad, double *value_host)
{
    tt_status st = reg_check(h, TT_F64, c, grad, value_host);
    if (st == TT_OK && !(delta > 0.0 && std::isfinite(delta))) { set_error("delta must be positive"); st = TT_INVALID_ARG; }
    return st != TT_OK ? st : tv_impl<double>(h, c, delta, grad, value_host);
}

}  // extern "C"
