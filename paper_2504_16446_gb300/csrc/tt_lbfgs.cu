// tt_lbfgs.cu -- device-resident L-BFGS (Section "Optimization"): two-loop
// recursion (Nocedal & Wright, Algorithm 7.4, H_0 = gamma I with gamma =
// s.y / y.y of the newest pair), backtracking Armijo line search.
//
// The recursion runs on the Gram matrix of its basis vectors instead of on
// the vectors themselves (the vector-free formulation of Chen, Wang & Zhou,
// NIPS 2014): every vector the two loops produce is a linear combination of
// b = (s_0 .. s_{m-1}, y_0 .. y_{m-1}, g), so each dot product they need is
// a combination of entries of the FP64 Gram matrix b_i . b_j, and the
// direction is d = -sum_i c_i b_i for coefficients computed on the host.
// Per iteration the vectors are touched by three kernels: one forms d and
// the first trial point, one forms the new pair s = x_t - x, y = g_t - g with
// its six dot products, one takes the dot products of the new pair and the
// new gradient with the stored pairs.  The recursion itself -- the same
// arithmetic as the two loops, in exact arithmetic -- costs O(m^2) on the
// host.  Dot products of float vectors use compensated FP32 accumulation
// (Dot2) within a CTA and FP64 across CTAs; double vectors use FP64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <utility>
#include <vector>

#include "tt_internal.cuh"

template <typename T>
tt_status tt_grad_enqueue(tt_handle *h, const T *c, const T *I, const T *W, T *g);
tt_status tt_read_loss(tt_handle *h, double *loss_host);

using namespace tt;

#define TT_CUDA(call, what)                                          \
    do {                                                             \
        cudaError_t _e = (call);                                     \
        if (_e != cudaSuccess) return ::tt::cuda_fail(_e, what);     \
    } while (0)

namespace {

constexpr int kMaxM = 64;

// Blocks of the per-element kernels (four elements per thread): a multiple of
// the SM count, capped.
unsigned elem_blocks(long long n)
{
    long long b = (n / 4 + 255) / 256;
    return (unsigned)std::max(1LL, std::min(b, 16LL * current_sm_count()));
}

// Four consecutive elements as one 16-byte access (two for double).  Every
// vector of the solver starts on a 256-byte boundary, so element 4q is
// 16-byte aligned.
__device__ __forceinline__ void ld4(const float *__restrict__ p, float (&v)[4])
{
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const double *__restrict__ p, double (&v)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float *__restrict__ p, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double *__restrict__ p, const double (&v)[4])
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// Block sum of a double, result on thread 0 (blockDim 256).
__device__ __forceinline__ double block_total(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

// Linear combination of up to 2 kMaxM + 1 vectors (kernel parameters).
template <typename T>
struct Combo {
    const T *v[2 * kMaxM + 1];
    double c[2 * kMaxM + 1];
    int n;
};

// d = sum_i c_i v_i (in T, coefficients rounded to T, summed in order i),
// xt = x + a d; four elements per thread and step, the last n % 4 elements
// by the first threads.
template <typename T>
__global__ void k_direction(const __grid_constant__ Combo<T> cb, const T *__restrict__ x, T *__restrict__ d,
                            T *__restrict__ xt, double a, long long n)
{
    const long long n4 = n / 4, stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T ta = (T)a;
    for (long long q = t0; q < n4; q += stride) {
        T s[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 4
        for (int i = 0; i < cb.n; ++i) {
            T v[4];
            ld4(cb.v[i] + 4 * q, v);
            const T ci = (T)cb.c[i];
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] = fma(ci, v[k], s[k]);
        }
        T xv[4], xn[4];
        ld4(x + 4 * q, xv);
#pragma unroll
        for (int k = 0; k < 4; ++k) xn[k] = xv[k] + ta * s[k];
        st4(d + 4 * q, s);
        st4(xt + 4 * q, xn);
    }
    if (t0 < n - 4 * n4) {
        const long long e = 4 * n4 + t0;
        T sv = T(0);
        for (int i = 0; i < cb.n; ++i) sv = fma((T)cb.c[i], cb.v[i][e], sv);
        d[e] = sv;
        xt[e] = x[e] + ta * sv;
    }
}

// Dot-product accumulator: compensated FP32 for float vectors, FP64 otherwise.
template <typename T>
struct Acc {
    double v = 0.0;
    __device__ void add(T x, T y) { v = fma(x, y, v); }
    __device__ double value() const { return v; }
};
template <>
struct Acc<float> {
    Dot2 a = {0.f, 0.f};
    __device__ void add(float x, float y) { dot2_add(a, x, y); }
    __device__ double value() const { return dot2_value(a); }
};

// CTA total of an accumulator (thread 0): FP64 tree for double, the
// compensated FP32 tree for float.
__device__ __forceinline__ double acc_total(const Acc<double> &a, double *red) { return block_total(a.value(), red); }
__device__ __forceinline__ double acc_total(const Acc<float> &a, double *red)
{
    return dot2_block_sum(a.a, reinterpret_cast<Dot2 *>(red));
}

// xt = x + a d
template <typename T>
__global__ void k_trial(const T *__restrict__ x, const T *__restrict__ d, T *__restrict__ xt, double a, long long n)
{
    const long long n4 = n / 4, stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const T ta = (T)a;
    for (long long q = t0; q < n4; q += stride) {
        T xv[4], dv[4];
        ld4(x + 4 * q, xv);
        ld4(d + 4 * q, dv);
#pragma unroll
        for (int k = 0; k < 4; ++k) xv[k] = xv[k] + ta * dv[k];
        st4(xt + 4 * q, xv);
    }
    if (t0 < n - 4 * n4) {
        const long long e = 4 * n4 + t0;
        xt[e] = x[e] + ta * d[e];
    }
}

// s = xt - x, y = gt - g (stored), and per-CTA partials of
// s.s, s.y, y.y, gt.s, gt.y, gt.gt at part[k * gridDim.x + blockIdx.x].
// Grid-stride over quads; the last CTA also takes the n % 4 tail.
template <typename T>
__global__ void k_pair(const T *__restrict__ x, const T *__restrict__ xt, const T *__restrict__ g,
                       const T *__restrict__ gt, T *__restrict__ s_out, T *__restrict__ y_out, long long n,
                       double *__restrict__ part)
{
    __shared__ double red[32];
    Acc<T> acc[6];
    auto one = [&](T s, T y, T gn) {
        acc[0].add(s, s);
        acc[1].add(s, y);
        acc[2].add(y, y);
        acc[3].add(gn, s);
        acc[4].add(gn, y);
        acc[5].add(gn, gn);
    };
    const long long n4 = n / 4, stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        T xv[4], xtv[4], gv[4], gtv[4], sv[4], yv[4];
        ld4(x + 4 * q, xv);
        ld4(xt + 4 * q, xtv);
        ld4(g + 4 * q, gv);
        ld4(gt + 4 * q, gtv);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sv[k] = xtv[k] - xv[k];
            yv[k] = gtv[k] - gv[k];
            one(sv[k], yv[k], gtv[k]);
        }
        st4(s_out + 4 * q, sv);
        st4(y_out + 4 * q, yv);
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x < n % 4) {
        const long long e = n - n % 4 + threadIdx.x;
        const T sv = xt[e] - x[e], yv = gt[e] - g[e];
        s_out[e] = sv;
        y_out[e] = yv;
        one(sv, yv, gt[e]);
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const double v = acc_total(acc[k], red);
        if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = v;
    }
}

// Dot products of the new pair (s, y) and the new gradient gt with stored
// pair j = slots[blockIdx.y]: s.S_j, s.Y_j, y.S_j, y.Y_j, gt.S_j, gt.Y_j.
template <typename T>
struct Slots {
    const T *S[kMaxM];
    const T *Y[kMaxM];
};

// CTA (b, p) takes stored pairs j = 2p and 2p + 1 (when it exists), so that
// s, y and gt are read once per two pairs; grid-stride over quads.
// Partials at part[(j * 6 + k) * gridDim.x + b].
template <typename T>
__global__ void k_cross(const __grid_constant__ Slots<T> sl, int nu, const T *__restrict__ s,
                        const T *__restrict__ y, const T *__restrict__ gt, long long n, double *__restrict__ part)
{
    __shared__ double red[32];
    const int j0 = 2 * blockIdx.y;
    const bool two = j0 + 1 < nu;
    const T *S0 = sl.S[j0], *Y0 = sl.Y[j0];
    const T *S1 = two ? sl.S[j0 + 1] : S0, *Y1 = two ? sl.Y[j0 + 1] : Y0;
    Acc<T> acc[12];
    auto one = [&](Acc<T> *a, T u, T w, T sv, T yv, T gv) {
        a[0].add(sv, u);
        a[1].add(sv, w);
        a[2].add(yv, u);
        a[3].add(yv, w);
        a[4].add(gv, u);
        a[5].add(gv, w);
    };
    const long long n4 = n / 4, stride = (long long)gridDim.x * blockDim.x;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        T sv[4], yv[4], gv[4], a0[4], b0[4];
        ld4(s + 4 * q, sv);
        ld4(y + 4 * q, yv);
        ld4(gt + 4 * q, gv);
        ld4(S0 + 4 * q, a0);
        ld4(Y0 + 4 * q, b0);
#pragma unroll
        for (int k = 0; k < 4; ++k) one(acc, a0[k], b0[k], sv[k], yv[k], gv[k]);
        if (two) {
            T a1[4], b1[4];
            ld4(S1 + 4 * q, a1);
            ld4(Y1 + 4 * q, b1);
#pragma unroll
            for (int k = 0; k < 4; ++k) one(acc + 6, a1[k], b1[k], sv[k], yv[k], gv[k]);
        }
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x < n % 4) {
        const long long e = n - n % 4 + threadIdx.x;
        one(acc, S0[e], Y0[e], s[e], y[e], gt[e]);
        if (two) one(acc + 6, S1[e], Y1[e], s[e], y[e], gt[e]);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        if (k >= 6 && !two) break;               // uniform across the CTA
        const double v = acc_total(acc[k], red);
        if (threadIdx.x == 0) part[((size_t)j0 * 6 + k) * gridDim.x + blockIdx.x] = v;
    }
}

// out[r] = sum of part[r * nb .. r * nb + nb) in a fixed order (one CTA per row).
__global__ void k_rows(const double *__restrict__ part, int nb, double *__restrict__ out)
{
    __shared__ double red[32];
    double v = 0.0;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) v += part[(size_t)blockIdx.x * nb + t];
    v = block_total(v, red);
    if (threadIdx.x == 0) out[blockIdx.x] = v;
}

}  // namespace

struct tt_lbfgs {
    tt_handle *h = nullptr;
    int m = 0;
    long long n = 0;
    void *slab = nullptr;         // one allocation holding every vector below
    void *x = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr, *ss = nullptr, *ys = nullptr;
    std::vector<void *> S, Y;
    int count = 0, head = -1;     // stored pairs; slot of the newest
    double f = 0.0;
    long long iterations = 0, evaluations = 1;   // accepted steps; gradient evaluations (creation's included)
    double last_step = 0.0;       // line-search step of the last accepted iteration, along d
    const void *I = nullptr, *W = nullptr;
    // Gram matrix of b = (S_0..S_{m-1}, Y_0..Y_{m-1}, g), (2m+1)^2, FP64
    std::vector<double> gram;
    double *part = nullptr;       // device partials
    double *dots = nullptr;       // device row sums
    double *pinned = nullptr;     // host copy of dots
    int pair_blocks = 0;          // CTAs of the pair / cross dot kernels (four per SM)
    int nb = 2 * kMaxM + 1;
    double &G(int i, int j) { return gram[(size_t)i * nb + j]; }
    int iS(int slot) const { return slot; }
    int iY(int slot) const { return m + slot; }
    int ig() const { return 2 * m; }
};

static void free_state(tt_lbfgs *st)
{
    if (!st) return;
    cudaFree(st->slab);
    cudaFree(st->part); cudaFree(st->dots);
    if (st->pinned) cudaFreeHost(st->pinned);
    delete st;
}

// Two-loop recursion on the Gram matrix: coefficients c of d = sum c_i b_i
// and g.d.  Without stored pairs d = -g.
static void direction_coeffs(tt_lbfgs *st, std::vector<double> &c, double &gd)
{
    const int nb = st->nb, m = st->m;
    c.assign(nb, 0.0);
    c[st->ig()] = 1.0;                                   // q = g
    std::vector<double> alpha(m, 0.0);
    auto dot_with = [&](int row) {                       // b_row . (sum c_i b_i)
        double v = 0.0;
        for (int i = 0; i < nb; ++i)
            if (c[i] != 0.0) v += c[i] * st->G(row, i);
        return v;
    };
    for (int t = 0; t < st->count; ++t) {               // newest -> oldest
        const int i = (st->head - t + m) % m;
        const double rho = 1.0 / st->G(st->iS(i), st->iY(i));
        alpha[i] = rho * dot_with(st->iS(i));
        c[st->iY(i)] -= alpha[i];
    }
    if (st->count > 0) {
        const int h = st->head;
        const double gamma = st->G(st->iS(h), st->iY(h)) / st->G(st->iY(h), st->iY(h));
        for (double &v : c) v *= gamma;
    }
    for (int t = st->count - 1; t >= 0; --t) {          // oldest -> newest
        const int i = (st->head - t + m) % m;
        const double rho = 1.0 / st->G(st->iS(i), st->iY(i));
        const double beta = rho * dot_with(st->iY(i));
        c[st->iS(i)] += alpha[i] - beta;
    }
    for (double &v : c) v = -v;                          // d = -r
    gd = dot_with(st->ig());
}

template <typename T>
static tt_status enqueue_direction(tt_lbfgs *st, const std::vector<double> &c, double a)
{
    tt_handle *h = st->h;
    Combo<T> cb;
    cb.n = 0;
    for (int i = 0; i < st->nb; ++i) {
        if (c[i] == 0.0) continue;
        const int m = st->m;
        cb.v[cb.n] = (const T *)(i == st->ig() ? st->g : (i < m ? st->S[i] : st->Y[i - m]));
        cb.c[cb.n] = c[i];
        ++cb.n;
    }
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_direction<T><<<elem_blocks(st->n), 256, 0, h->stream>>>(cb, (const T *)st->x, (T *)st->d, (T *)st->xt, a,
                                                             st->n);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    TT_CUDA(e, "lbfgs direction");
    return TT_OK;
}

template <typename T>
static tt_status enqueue_trial(tt_lbfgs *st, double a)
{
    tt_handle *h = st->h;
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_trial<T><<<elem_blocks(st->n), 256, 0, h->stream>>>((const T *)st->x, (const T *)st->d, (T *)st->xt, a, st->n);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    TT_CUDA(e, "lbfgs trial point");
    return TT_OK;
}

// Stored pair slots, newest first.
static std::vector<int> used_slots(const tt_lbfgs *st)
{
    std::vector<int> used;
    for (int t = 0; t < st->count; ++t) used.push_back((st->head - t + st->m) % st->m);
    return used;
}

// For a trial point: its pair s = xt - x, y = gt - g into scratch, the six
// dot products of the pair and gt, and those of s, y, gt with every stored
// pair; their copy to the host is enqueued behind them, so the stream
// synchronisation that reads the trial loss also delivers them.  (Enqueued
// before the Armijo test is known: a rejected trial wastes these kernels,
// an accepted one -- nearly every first trial -- saves a synchronisation.)
template <typename T>
static tt_status enqueue_pair_dots(tt_lbfgs *st, const std::vector<int> &used)
{
    tt_handle *h = st->h;
    const int nu = (int)used.size();
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_pair<T><<<st->pair_blocks, 256, 0, h->stream>>>((const T *)st->x, (const T *)st->xt, (const T *)st->g,
                                                (const T *)st->gt, (T *)st->ss, (T *)st->ys, st->n, st->part);
    if (nu > 0) {
        Slots<T> sl;
        for (int u = 0; u < nu; ++u) { sl.S[u] = (const T *)st->S[used[u]]; sl.Y[u] = (const T *)st->Y[used[u]]; }
        k_cross<T><<<dim3(st->pair_blocks, (nu + 1) / 2), 256, 0, h->stream>>>(
            sl, nu, (const T *)st->ss, (const T *)st->ys, (const T *)st->gt, st->n, st->part + 6 * st->pair_blocks);
    }
    const int rows = 6 + 6 * nu;
    k_rows<<<rows, 256, 0, h->stream>>>(st->part, st->pair_blocks, st->dots);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    TT_CUDA(e, "lbfgs pair dots");
    TT_CUDA(cudaMemcpyAsync(st->pinned, st->dots, sizeof(double) * rows, cudaMemcpyDeviceToHost, h->stream),
            "lbfgs dots copy");
    return TT_OK;
}

// Accepted trial (its dot products have arrived in st->pinned): the Gram
// matrix is updated, the pair stored if the curvature condition holds, and
// x, g advance.
static void finish_accept(tt_lbfgs *st, const std::vector<int> &used)
{
    const int m = st->m;
    const int nu = (int)used.size();
    const double *P = st->pinned;
    const double ss = P[0], sy = P[1], yy = P[2], gs = P[3], gy = P[4], gg = P[5];
    const int ig = st->ig();
    // new gradient against the stored pairs
    for (int u = 0; u < nu; ++u) {
        const int j = used[u];
        st->G(ig, st->iS(j)) = st->G(st->iS(j), ig) = P[6 + 6 * u + 4];
        st->G(ig, st->iY(j)) = st->G(st->iY(j), ig) = P[6 + 6 * u + 5];
    }
    st->G(ig, ig) = gg;
    if (sy > 1e-10 * std::sqrt(ss) * std::sqrt(yy)) {
        const int k = (st->head + 1) % m;                 // slot of the new pair (oldest one if full)
        std::swap(st->S[k], st->ss);
        std::swap(st->Y[k], st->ys);
        if (st->count < m) ++st->count;
        st->head = k;
        const int sk = st->iS(k), yk = st->iY(k);
        for (int u = 0; u < nu; ++u) {
            const int j = used[u];
            if (j == k) continue;                          // the replaced pair
            const double *r = P + 6 + 6 * u;
            st->G(sk, st->iS(j)) = st->G(st->iS(j), sk) = r[0];
            st->G(sk, st->iY(j)) = st->G(st->iY(j), sk) = r[1];
            st->G(yk, st->iS(j)) = st->G(st->iS(j), yk) = r[2];
            st->G(yk, st->iY(j)) = st->G(st->iY(j), yk) = r[3];
        }
        st->G(sk, sk) = ss;
        st->G(sk, yk) = st->G(yk, sk) = sy;
        st->G(yk, yk) = yy;
        st->G(ig, sk) = st->G(sk, ig) = gs;
        st->G(ig, yk) = st->G(yk, ig) = gy;
    }
    std::swap(st->x, st->xt);
    std::swap(st->g, st->gt);
}


template <typename T>
static tt_status lbfgs_step(tt_lbfgs *st, double *loss_out, int *n_evals_out)
{
    tt_handle *h = st->h;
    std::vector<double> c;
    double gd = 0.0;
    direction_coeffs(st, c, gd);
    double step0 = 1.0;
    if (st->count > 0 && !(gd < 0.0)) {                  // not a descent direction: clear the memory
        st->count = 0;
        st->head = -1;
        direction_coeffs(st, c, gd);
    }
    if (st->count == 0) {
        const double gg = st->G(st->ig(), st->ig());
        if (!(gg > 0.0) || !std::isfinite(gg)) {
            // stationary point (or non-finite gradient): nothing to do
            if (loss_out) *loss_out = st->f;
            if (n_evals_out) *n_evals_out = 0;
            if (!std::isfinite(gg)) { set_error("gradient is not finite"); return TT_NONFINITE; }
            return TT_OK;
        }
        step0 = 1.0 / std::sqrt(gg);
        gd = -gg;
    }

    const double c1 = 1e-4;
    const int max_evals = 20;
    double a = step0;
    tt_status s = enqueue_direction<T>(st, c, a);
    if (s != TT_OK) return s;
    const std::vector<int> used = used_slots(st);
    for (int ne = 1; ne <= max_evals; ++ne) {
        if (ne > 1) {
            s = enqueue_trial<T>(st, a);
            if (s != TT_OK) return s;
        }
        s = tt_grad_enqueue<T>(h, (const T *)st->xt, (const T *)st->I, (const T *)st->W, (T *)st->gt);
        if (s != TT_OK) return s;
        s = enqueue_pair_dots<T>(st, used);
        if (s != TT_OK) return s;
        double ft = 0.0;
        s = tt_read_loss(h, &ft);                        // synchronises: the dots are in too
        ++st->evaluations;
        if (s != TT_OK && s != TT_NONFINITE) return s;
        if (s == TT_OK && ft <= st->f + c1 * a * gd) {
            finish_accept(st, used);
            st->f = ft;
            ++st->iterations;
            st->last_step = a;
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

template <typename T>
static tt_status initial_gram(tt_lbfgs *st)
{
    tt_handle *h = st->h;
    TT_CUDA((vec_dot<T>(h, (const T *)st->g, (const T *)st->g, st->n, st->part, st->dots, nullptr, 1.0)),
            "lbfgs g.g");
    TT_CUDA(cudaMemcpyAsync(st->pinned, st->dots, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "copy");
    TT_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    st->G(st->ig(), st->ig()) = st->pinned[0];
    return TT_OK;
}

// Memory of a state: every vector in one slab of 256-byte aligned pitches
// (x, g, d, xt, gt, scratch pair, m stored pairs), the dot-product partials
// and their pinned host copy.  Counters and the Gram matrix start empty.
static tt_status alloc_state(tt_handle *h, int m, const void *I, const void *W, tt_lbfgs **out)
{
    tt_lbfgs *st = new tt_lbfgs();
    st->h = h;
    st->m = m;
    st->nb = 2 * m + 1;
    st->gram.assign((size_t)st->nb * st->nb, 0.0);
    st->n = h->nvox() * h->K;
    st->I = I;
    st->W = W;
    const size_t bytes = h->esize() * st->n;
    const size_t pitch = (bytes + 255) / 256 * 256;
    cudaError_t e = cudaMalloc(&st->slab, pitch * (7 + 2 * (size_t)m));
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "L-BFGS state: cudaMalloc"); }
    char *base = (char *)st->slab;
    void **bufs[] = {&st->x, &st->g, &st->d, &st->xt, &st->gt, &st->ss, &st->ys};
    for (void **b : bufs) { *b = base; base += pitch; }
    st->S.assign(m, nullptr);
    st->Y.assign(m, nullptr);
    for (int i = 0; i < m; ++i) {
        st->S[i] = base; base += pitch;
        st->Y[i] = base; base += pitch;
    }
    const size_t rows = 6 + 6 * (size_t)m;
    st->pair_blocks = 4 * h->n_sm;
    e = cudaMalloc(&st->part, sizeof(double) * std::max<size_t>(rows * st->pair_blocks, dot_blocks(h)));
    if (e == cudaSuccess) e = cudaMalloc(&st->dots, sizeof(double) * rows);
    if (e == cudaSuccess) e = cudaMallocHost(&st->pinned, sizeof(double) * rows);
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "L-BFGS state"); }
    *out = st;
    return TT_OK;
}

// Checkpoint layout: this header, the Gram matrix (nb x nb FP64), then x, g
// and the stored pairs S, Y from the newest to the oldest, each n elements
// of the handle's element type.
static const char kCheckpointMagic[8] = {'T', 'T', 'L', 'B', 'F', 'G', 'S', '1'};
struct CheckpointHeader {
    char magic[8];
    int32_t m, count, head, esize;
    int64_t n;
    double f;
    int32_t nb, reserved;
    int64_t iterations, evaluations;
    double last_step;
};

static size_t checkpoint_bytes(int nb, long long n, size_t esize, int count)
{
    return sizeof(CheckpointHeader) + sizeof(double) * (size_t)nb * nb + esize * (size_t)n * (2 + 2 * (size_t)count);
}

extern "C" {

tt_status tt_lbfgs_create(tt_handle *h, int m, const void *c0, const void *I, const void *W, tt_lbfgs **out)
{
    if (!out) { set_error("tt_lbfgs_create: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (!h || !I || m < 1 || m > kMaxM) {
        set_error("tt_lbfgs_create: need a handle, I and 1 <= m <= 64");
        return TT_INVALID_ARG;
    }
    tt_lbfgs *st = nullptr;
    tt_status s = alloc_state(h, m, I, W, &st);
    if (s != TT_OK) return s;
    // c0 == NULL: start at zero, where the evaluation needs no forward march
    const size_t bytes = h->esize() * st->n;
    cudaError_t e = c0 ? cudaMemcpyAsync(st->x, c0, bytes, cudaMemcpyDeviceToDevice, h->stream)
                       : cudaMemsetAsync(st->x, 0, bytes, h->stream);
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_create"); }
    const void *xc = c0 ? st->x : nullptr;
    s = (h->prec != TT_F64)
            ? tt_grad_enqueue<float>(h, (const float *)xc, (const float *)I, (const float *)W, (float *)st->g)
            : tt_grad_enqueue<double>(h, (const double *)xc, (const double *)I, (const double *)W, (double *)st->g);
    if (s == TT_OK) s = tt_read_loss(h, &st->f);
    if (s == TT_OK) s = (h->prec != TT_F64) ? initial_gram<float>(st) : initial_gram<double>(st);
    if (s != TT_OK) { free_state(st); return s; }
    *out = st;
    return TT_OK;
}

}  // extern "C"

// The loss is quadratic along any ray: L(a u) = a^2 q - 2 a l + L0 with
// q = |A u|^2_W and l = <A u, W I>.  The gradient at zero, g0 = -2 A^T W I,
// gives l = -<u, g0> / 2, and one evaluation at u gives q = L(u) - L0 + 2 l
// and g(u) = 2 A^T W A u + g0.  The minimiser a* = l / q, its loss
// L0 - l^2 / q and its gradient a* g(u) + (1 - a*) g0 follow without an
// evaluation at a* u.
template <typename T>
static tt_status create_ray(tt_handle *h, int m, const T *u, const T *g0, double L0, const void *I, const void *W,
                            double *alpha_out, tt_lbfgs **out)
{
    tt_lbfgs *st = nullptr;
    tt_status s = alloc_state(h, m, I, W, &st);
    if (s != TT_OK) return s;
    T *x = (T *)st->x, *g = (T *)st->g;
    const size_t bytes = h->esize() * st->n;
    double Lu = 0.0;
    s = tt_grad_enqueue<T>(h, u, (const T *)I, (const T *)W, g);
    cudaError_t e = cudaSuccess;
    if (s == TT_OK) e = vec_dot<T>(h, u, g0, st->n, st->part, st->dots, nullptr, 1.0);
    if (s == TT_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(st->pinned, st->dots, sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (s == TT_OK && e != cudaSuccess) s = cuda_fail(e, "tt_lbfgs_create_ray: <u, g0>");
    if (s == TT_OK) s = tt_read_loss(h, &Lu);   // synchronises: the dot product is in st->pinned too
    if (s != TT_OK) { free_state(st); return s; }
    const double lin = -0.5 * st->pinned[0];
    const double quad = Lu - L0 + 2.0 * lin;
    double alpha = 0.0, f = L0;
    if (quad > 0.0 && std::isfinite(quad) && std::isfinite(lin)) {
        alpha = lin / quad;
        f = L0 - lin * lin / quad;
    }
    if (alpha != 0.0 && f < L0) {
        e = vec_axpby<T>(h, x, u, st->n, alpha, nullptr, 0.0);                    // x = a* u
        if (e == cudaSuccess) e = vec_axpby<T>(h, g, g0, st->n, 1.0 - alpha, nullptr, alpha);   // g = a* g(u) + (1 - a*) g0
    } else {
        alpha = 0.0;
        f = L0;
        e = cudaMemsetAsync(x, 0, bytes, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(g, g0, bytes, cudaMemcpyDeviceToDevice, h->stream);
    }
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_create_ray: start point"); }
    st->f = f;
    s = initial_gram<T>(st);
    if (s != TT_OK) { free_state(st); return s; }
    if (alpha_out) *alpha_out = alpha;
    *out = st;
    return TT_OK;
}

extern "C" {

tt_status tt_lbfgs_create_ray(tt_handle *h, int m, const void *u, const void *g0, double loss0, const void *I,
                              const void *W, double *alpha_out, tt_lbfgs **out)
{
    if (!out) { set_error("tt_lbfgs_create_ray: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (!h || !u || !g0 || !I || m < 1 || m > kMaxM || !std::isfinite(loss0) || loss0 < 0.0) {
        set_error("tt_lbfgs_create_ray: need a handle, u, g0, I, a finite loss0 >= 0 and 1 <= m <= 64");
        return TT_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(g0) & 15u) != 0) {
        set_error("tt_lbfgs_create_ray: g0 must be 16-byte aligned");
        return TT_INVALID_ARG;
    }
    return (h->prec != TT_F64)
               ? create_ray<float>(h, m, (const float *)u, (const float *)g0, loss0, I, W, alpha_out, out)
               : create_ray<double>(h, m, (const double *)u, (const double *)g0, loss0, I, W, alpha_out, out);
}

tt_status tt_lbfgs_stats(const tt_lbfgs *st, long long *iterations, long long *evaluations, double *last_step)
{
    if (!st) { set_error("tt_lbfgs_stats: null state"); return TT_INVALID_ARG; }
    if (iterations) *iterations = st->iterations;
    if (evaluations) *evaluations = st->evaluations;
    if (last_step) *last_step = st->last_step;
    return TT_OK;
}

long long tt_lbfgs_checkpoint_bytes(const tt_lbfgs *st)
{
    if (!st) return 0;
    return (long long)checkpoint_bytes(st->nb, st->n, st->h ? st->h->esize() : 0, st->count);
}

tt_status tt_lbfgs_save(tt_handle *h, const tt_lbfgs *st, void *buf, long long bytes)
{
    if (!h || !st || st->h != h) { set_error("tt_lbfgs_save: state does not belong to this handle"); return TT_INVALID_ARG; }
    const size_t es = h->esize(), need = checkpoint_bytes(st->nb, st->n, es, st->count);
    if (!buf || bytes < (long long)need) {
        set_error("tt_lbfgs_save: buf must hold tt_lbfgs_checkpoint_bytes(st) bytes");
        return TT_INVALID_ARG;
    }
    CheckpointHeader hd{};
    std::memcpy(hd.magic, kCheckpointMagic, sizeof hd.magic);
    hd.m = st->m; hd.count = st->count; hd.head = st->head; hd.esize = (int)es;
    hd.n = st->n; hd.f = st->f; hd.nb = st->nb;
    hd.iterations = st->iterations; hd.evaluations = st->evaluations; hd.last_step = st->last_step;
    char *p = (char *)buf;
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    std::memcpy(p, st->gram.data(), sizeof(double) * st->gram.size());
    p += sizeof(double) * st->gram.size();
    const size_t vb = es * st->n;
    std::vector<const void *> src = {st->x, st->g};
    for (int t = 0; t < st->count; ++t) {
        const int k = (st->head - t + st->m) % st->m;
        src.push_back(st->S[k]);
        src.push_back(st->Y[k]);
    }
    for (const void *v : src) {
        TT_CUDA(cudaMemcpyAsync(p, v, vb, cudaMemcpyDeviceToHost, h->stream), "tt_lbfgs_save: copy");
        p += vb;
    }
    TT_CUDA(cudaStreamSynchronize(h->stream), "tt_lbfgs_save: synchronize");
    return TT_OK;
}

tt_status tt_lbfgs_restore(tt_handle *h, const void *buf, long long bytes, const void *I, const void *W, tt_lbfgs **out)
{
    if (!out) { set_error("tt_lbfgs_restore: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (!h || !buf || !I || bytes < (long long)sizeof(CheckpointHeader)) {
        set_error("tt_lbfgs_restore: need a handle, a checkpoint and I");
        return TT_INVALID_ARG;
    }
    CheckpointHeader hd;
    std::memcpy(&hd, buf, sizeof hd);
    const size_t es = h->esize();
    if (std::memcmp(hd.magic, kCheckpointMagic, sizeof hd.magic) != 0 || hd.m < 1 || hd.m > kMaxM ||
        hd.nb != 2 * hd.m + 1 || hd.count < 0 || hd.count > hd.m || (hd.count > 0 && (hd.head < 0 || hd.head >= hd.m)) ||
        hd.n != h->nvox() * h->K || hd.esize != (int)es ||
        bytes != (long long)checkpoint_bytes(hd.nb, hd.n, es, hd.count)) {
        set_error("tt_lbfgs_restore: not a checkpoint of an L-BFGS state of this problem and precision");
        return TT_INVALID_ARG;
    }
    tt_lbfgs *st = nullptr;
    tt_status s = alloc_state(h, hd.m, I, W, &st);
    if (s != TT_OK) return s;
    st->count = hd.count;
    st->head = hd.head;
    st->f = hd.f;
    st->iterations = hd.iterations;
    st->evaluations = hd.evaluations;
    st->last_step = hd.last_step;
    const char *p = (const char *)buf + sizeof hd;
    std::memcpy(st->gram.data(), p, sizeof(double) * st->gram.size());
    p += sizeof(double) * st->gram.size();
    const size_t vb = es * st->n;
    std::vector<void *> dst = {st->x, st->g};
    for (int t = 0; t < st->count; ++t) {
        const int k = (st->head - t + st->m) % st->m;
        dst.push_back(st->S[k]);
        dst.push_back(st->Y[k]);
    }
    cudaError_t e = cudaSuccess;
    for (void *v : dst) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(v, p, vb, cudaMemcpyHostToDevice, h->stream);
        p += vb;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) { free_state(st); return cuda_fail(e, "tt_lbfgs_restore: copy"); }
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
