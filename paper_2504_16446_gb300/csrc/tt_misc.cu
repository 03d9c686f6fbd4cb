// tt_misc.cu -- layout, reduction, vector and basis-matrix kernels of libtt.
#include <cmath>

#include "tt_kernels.cuh"

namespace tt {

// ------------------------------------------------------------- layout

// Interior of the padded volume: cpad[x+2][y+2][z+2][i] = c[x][y][z][i] for
// i < K, 0 for K <= i < KP (the two-voxel border is zeroed once at creation);
// with cpadx, also the x-innermost copy cpadx[z+2][y+2][x+2][i].
// One thread per 4-channel chunk of a voxel: consecutive threads read
// consecutive chunks of c and write consecutive 16-byte (8-byte for 2-byte
// storage) pieces of cpad rows.  Index arithmetic is 32-bit (tt_create caps
// the volume at 2^24 voxels).
template <typename S>
__device__ __forceinline__ void store4(S *p, float a, float b, float c, float d)
{
    if constexpr (std::is_same<S, float>::value) {
        *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2(pack2(a, b, (S *)nullptr), pack2(c, d, (S *)nullptr));
    }
}

template <typename T, typename S>
__global__ void k_pack(const T *__restrict__ c, S *__restrict__ cpad, S *__restrict__ cpadx, int nx, int ny, int nz,
                       int K, int KP)
{
    const int QP = KP / 4;
    const int n = nx * ny * nz * QP;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int v = t / QP, i0 = 4 * (t - v * QP);
        const int z = v % nz, xy = v / nz, y = xy % ny, x = xy / ny;
        const T *src = c + (long long)v * K;
        T val[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) val[i] = i0 + i < K ? __ldg(src + i0 + i) : T(0);
        S *dst = cpad + (((long long)(x + 2) * (ny + 4) + (y + 2)) * (nz + 4) + (z + 2)) * KP + i0;
        S *dstx = cpadx ? cpadx + (((long long)(z + 2) * (ny + 4) + (y + 2)) * (nx + 4) + (x + 2)) * KP + i0 : nullptr;
        if constexpr (std::is_same<T, double>::value) {
            reinterpret_cast<double2 *>(dst)[0] = make_double2(val[0], val[1]);
            reinterpret_cast<double2 *>(dst)[1] = make_double2(val[2], val[3]);
            if (dstx) {
                reinterpret_cast<double2 *>(dstx)[0] = make_double2(val[0], val[1]);
                reinterpret_cast<double2 *>(dstx)[1] = make_double2(val[2], val[3]);
            }
        } else {
            store4<S>(dst, val[0], val[1], val[2], val[3]);
            if (dstx) store4<S>(dstx, val[0], val[1], val[2], val[3]);
        }
    }
}

template <typename T>
__global__ void k_unpack(const T *__restrict__ gpad, T *__restrict__ g, long long nvox, int K, int KP)
{
    const long long n = nvox * K;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / K;
        const int i = (int)(t - v * K);
        g[t] = __ldg(gpad + v * KP + i);
    }
}

static unsigned grid_for(long long n, int per_block = 256)
{
    long long b = (n + per_block - 1) / per_block;
    const long long cap = 32LL * current_sm_count();
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <typename T, typename S>
cudaError_t launch_pack(tt_handle *h, const T *c)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_PACK, &ev);
    S *cpadx = h->xcopy ? (S *)h->cpad + h->pad_vox * h->KP : nullptr;
    k_pack<T, S><<<grid_for(h->nvox() * h->KP / 4), 256, 0, h->stream>>>(c, (S *)h->cpad, cpadx, h->N[0], h->N[1],
                                                                       h->N[2], h->K, h->KP);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_PACK, ev);
    return e;
}

template <typename T>
cudaError_t launch_unpack(tt_handle *h, const T *gpad, T *g)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_UNPACK, &ev);
    k_unpack<T><<<grid_for(h->nvox() * h->K), 256, 0, h->stream>>>(gpad, g, h->nvox(), h->K, h->KP);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_UNPACK, ev);
    return e;
}

template cudaError_t launch_pack<float, float>(tt_handle *, const float *);
template cudaError_t launch_pack<double, double>(tt_handle *, const double *);
template cudaError_t launch_pack<float, __nv_bfloat16>(tt_handle *, const float *);
template cudaError_t launch_pack<float, __half>(tt_handle *, const float *);
template cudaError_t launch_unpack<float>(tt_handle *, const float *, float *);
template cudaError_t launch_unpack<double>(tt_handle *, const double *, double *);

// ------------------------------------------------------------- reductions

// out[0] = (add ? add[0] : 0) + mul * sum(partials[0..n)), summed in the
// fixed order of sum_fixed_order (the same as the loss reduction that the
// adjoint's first CTA performs).
__global__ void k_reduce(const double *__restrict__ partials, long long n, double *__restrict__ out,
                         const double *__restrict__ add, double mul)
{
    __shared__ double red[32];
    const double v = sum_fixed_order(partials, n, red);
    if (threadIdx.x == 0) out[0] = (add ? add[0] : 0.0) + mul * v;
}

cudaError_t launch_reduce(tt_handle *h, const double *partials, long long n, double *out, const double *add,
                          double mul)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_REDUCE, &ev);
    k_reduce<<<1, kThreads, 0, h->stream>>>(partials, n, out, add, mul);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_REDUCE, ev);
    return e;
}

// ------------------------------------------------------------- vectors

template <typename T>
__global__ void k_dot_partial(const T *__restrict__ x, const T *__restrict__ y, long long n,
                              double *__restrict__ partials)
{
    __shared__ double red[32];
    double v = 0.0;
    if constexpr (std::is_same<T, float>::value) {
        Dot2 a = {0.f, 0.f};                   // compensated FP32 per thread and across the CTA
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x)
            dot2_add(a, x[t], y[t]);
        v = dot2_block_sum(a, reinterpret_cast<Dot2 *>(red));
    } else {
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x)
            v = fma(x[t], y[t], v);
        v = block_sum(v, red);
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

template <typename T>
__global__ void k_axpby(T *__restrict__ y, const T *__restrict__ x, long long n, double ha,
                        const double *__restrict__ da, double hb)
{
    const T a = (T)(ha * (da ? da[0] : 1.0));
    const T b = (T)hb;
    // b == 0 overwrites y without reading it (y may hold NaN bit patterns).
    if (hb == 0.0) {
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x)
            y[t] = a * x[t];
    } else {
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
             t += (long long)gridDim.x * blockDim.x)
            y[t] = fma(a, x[t], b * y[t]);
    }
}

template <typename T>
__global__ void k_sub(T *__restrict__ out, const T *__restrict__ x, const T *__restrict__ y, long long n)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        out[t] = x[t] - y[t];
}

template <typename T>
cudaError_t vec_dot(tt_handle *h, const T *x, const T *y, long long n, double *partials, double *out,
                    const double *add, double mul)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_dot_partial<T><<<dot_blocks(h), 256, 0, h->stream>>>(x, y, n, partials);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    if (e != cudaSuccess) return e;
    return launch_reduce(h, partials, dot_blocks(h), out, add, mul);
}

template <typename T>
cudaError_t vec_axpby(tt_handle *h, T *y, const T *x, long long n, double ha, const double *da, double hb)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_axpby<T><<<grid_for(n), 256, 0, h->stream>>>(y, x, n, ha, da, hb);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    return e;
}

template <typename T>
cudaError_t vec_sub(tt_handle *h, T *out, const T *x, const T *y, long long n)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_VECTOR, &ev);
    k_sub<T><<<grid_for(n), 256, 0, h->stream>>>(out, x, y, n);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_VECTOR, ev);
    return e;
}

template cudaError_t vec_dot<float>(tt_handle *, const float *, const float *, long long, double *, double *,
                                    const double *, double);
template cudaError_t vec_dot<double>(tt_handle *, const double *, const double *, long long, double *,
                                     double *, const double *, double);
template cudaError_t vec_axpby<float>(tt_handle *, float *, const float *, long long, double, const double *,
                                      double);
template cudaError_t vec_axpby<double>(tt_handle *, double *, const double *, long long, double,
                                       const double *, double);
template cudaError_t vec_sub<float>(tt_handle *, float *, const float *, const float *, long long);
template cudaError_t vec_sub<double>(tt_handle *, double *, const double *, const double *, long long);

// ------------------------------------------------------------- real SH

// Even-l real SH at a direction (need not be normalised), written to
// out[i*stride].  Cartesian recurrences: with r = |q|, (x + i y)^m gives
// sin^m(theta) cos(m phi) and sin^m(theta) sin(m phi); the associated
// Legendre factor without its sin^m(theta) is the polynomial
//   Q_m^m = (2m-1)!!,  Q_{m+1}^m = (2m+1) z Q_m^m,
//   (l-m) Q_l^m = (2l-1) z Q_{l-1}^m - (l+m-1) Q_{l-2}^m
// and Y_lm = sqrt(2) N_lm Q_l^m Re/Im (x+iy)^m (m != 0), Y_l0 = N_l0 Q_l^0 with
// N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) -- orthonormal, no Condon-Shortley
// phase, polar axis +z (Section "Basis sets", SH).
template <typename T>
__device__ void sh_even(int L, T x, T y, T z, T *out, int stride)
{
    const T rn = T(1) / sqrt(x * x + y * y + z * z);
    x *= rn; y *= rn; z *= rn;
    T cr = T(1), ci = T(0);                 // (x + i y)^m
    T qmm = T(1);                           // Q_m^m
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            const T ncr = cr * x - ci * y, nci = cr * y + ci * x;
            cr = ncr; ci = nci;
            qmm *= T(2 * m - 1);
        }
        T q_lm2 = T(0), q_lm1 = qmm;        // Q_{l-2}^m, Q_{l-1}^m as l advances
        for (int l = m; l <= L; ++l) {
            T qlm;
            if (l == m) qlm = qmm;
            else if (l == m + 1) qlm = T(2 * m + 1) * z * qmm;
            else qlm = (T(2 * l - 1) * z * q_lm1 - T(l + m - 1) * q_lm2) / T(l - m);
            if (l > m) { q_lm2 = q_lm1; q_lm1 = qlm; }
            if ((l & 1) == 0) {
                // (l-m)!/(l+m)!
                T ratio = T(1);
                for (int t = l - m + 1; t <= l + m; ++t) ratio /= T(t);
                const T nlm = sqrt(T(2 * l + 1) / T(4.0 * M_PI) * ratio);
                const int base = l * (l - 1) / 2 + l;   // index of (l, m = 0)
                if (m == 0) {
                    out[base * stride] = nlm * qlm;
                } else {
                    const T f = T(M_SQRT2) * nlm * qlm;
                    out[(base + m) * stride] = f * cr;
                    out[(base - m) * stride] = f * ci;
                }
            }
        }
    }
}

// B[s][c][i] = 0.5 * sum_n w_n Y_i(R_s^T q(phi_n)), phi_n = mid + half x_n
// (Gauss-Legendre on the segment; 1/dphi * half = 0.5), Eq. (projection_matrix).
// One CTA per (c, s), one thread per quadrature node.
__global__ void __launch_bounds__(kQuadNodes)
k_basis(const double *__restrict__ frames /*[S][9]: p_s, q0_s, q90_s*/, const double *__restrict__ seg0,
        const double *__restrict__ seg1, const double *__restrict__ nodes, const double *__restrict__ weights,
        double cth, double sth, int L, int K, int C, double *__restrict__ B)
{
    extern __shared__ double ysh[];   // [kQuadNodes][K]
    const int c = blockIdx.x, s = blockIdx.y, t = threadIdx.x;
    const double *F = frames + 9 * s;
    const double half = 0.5 * (seg1[c] - seg0[c]), mid = 0.5 * (seg1[c] + seg0[c]);
    const double phi = mid + half * nodes[t];
    double sp, cp;
    sincos(phi, &sp, &cp);
    double q[3];
    for (int r = 0; r < 3; ++r) q[r] = cth * (cp * F[3 + r] + sp * F[6 + r]) - sth * F[r];
    sh_even<double>(L, q[0], q[1], q[2], ysh + t * K, 1);
    const double wt = 0.5 * weights[t];
    for (int i = 0; i < K; ++i) ysh[t * K + i] *= wt;
    __syncthreads();
    for (int i = t; i < K; i += blockDim.x) {
        double acc = 0.0;
        for (int n = 0; n < kQuadNodes; ++n) acc += ysh[n * K + i];
        B[((long long)s * C + c) * K + i] = acc;
    }
}

// Element-type basis matrix, zero padded to [S][CP][KP].
template <typename T>
__global__ void k_cast_basis(const double *__restrict__ B, T *__restrict__ Bp, int S, int C, int K, int CP, int KP)
{
    const long long n = (long long)S * CP * KP;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t % KP);
        const int c = (int)((t / KP) % CP);
        const int s = (int)(t / ((long long)KP * CP));
        Bp[t] = (i < K && c < C) ? (T)B[((long long)s * C + c) * K + i] : T(0);
    }
}

cudaError_t launch_basis(tt_handle *h, const double *nodes, const double *weights)
{
    // frames, segments: staged right after the node tables by the caller
    const double *frames = weights + kQuadNodes;
    const double *seg0 = frames + 9 * h->S;
    const double *seg1 = seg0 + h->C;
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_BASIS, &ev);
    const double th = 0.5 * h->two_theta;
    k_basis<<<dim3(h->C, h->S), kQuadNodes, kQuadNodes * h->K * sizeof(double), h->stream>>>(
        frames, seg0, seg1, nodes, weights, std::cos(th), std::sin(th), h->L, h->K, h->C, h->B64);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_BASIS, ev);
    return e;
}

template <typename T>
cudaError_t launch_cast_basis(tt_handle *h)
{
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_BASIS, &ev);
    k_cast_basis<T><<<grid_for((long long)h->S * h->CP * h->KP), 256, 0, h->stream>>>(
        h->B64, (T *)h->Bp, h->S, h->C, h->K, h->CP, h->KP);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_BASIS, ev);
    return e;
}
template cudaError_t launch_cast_basis<float>(tt_handle *);
template cudaError_t launch_cast_basis<double>(tt_handle *);

// c_lm = a_l sqrt(4 pi/(2l+1)) Y_lm(n): zonal function of axis n (addition theorem).
__global__ void k_zonal(int L, int K, long long n, const float *__restrict__ dirs, const float *__restrict__ amps,
                        float *__restrict__ c)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        float *out = c + t * K;
        sh_even<float>(L, dirs[3 * t], dirs[3 * t + 1], dirs[3 * t + 2], out, 1);
        const float *a = amps + t * (L / 2 + 1);
        for (int l = 0; l <= L; l += 2) {
            const float f = a[l / 2] * sqrtf(4.0f * (float)M_PI / (2 * l + 1));
            const int base = l * (l - 1) / 2;
            for (int i = 0; i < 2 * l + 1; ++i) out[base + i] *= f;
        }
    }
}

}  // namespace tt

extern "C" tt_status tt_zonal_to_sh(int ell_max, long long n, const float *dirs_dev, const float *amps_dev,
                                    float *c_dev, void *stream)
{
    if (ell_max < 0 || ell_max > tt::kMaxEll || (ell_max & 1) || n < 0) {
        tt::set_error("tt_zonal_to_sh: ell_max must be even in [0, 12] and n >= 0");
        return TT_INVALID_ARG;
    }
    if (n == 0) return TT_OK;
    if (!dirs_dev || !amps_dev || !c_dev) {
        tt::set_error("tt_zonal_to_sh: null pointer");
        return TT_INVALID_ARG;
    }
    tt::k_zonal<<<tt::grid_for(n), 256, 0, (cudaStream_t)stream>>>(ell_max, tt::num_coeffs(ell_max), n, dirs_dev,
                                                                   amps_dev, c_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return tt::cuda_fail(e, "tt_zonal_to_sh launch");
    return TT_OK;
}
