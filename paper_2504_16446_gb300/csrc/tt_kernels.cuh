// tt_kernels.cuh -- projector kernels of libtt (templates; instantiated per
// element type in tt_proj_f32.cu / tt_proj_f64.cu).
//
// Data layout in HBM (all row-major):
//   cpad [nx][ny][nz][KP]          coefficient volume, channel innermost, zero padded
//   Bp   [S][CP][KP]               basis matrix in the element type, zero padded
//   G    [S][nj][nk][KP]           back-contracted weighted residual, 2 B_s^T (W r)
//   gpad [nx][ny][nz][KP]          gradient / adjoint volume
// A lane group of LG consecutive lanes owns one ray (forward) or one voxel
// (adjoint); lane q of the group holds channels [q*CPL, (q+1)*CPL), so that a
// bilinear tap is one contiguous KP-element row read by LG lanes with 16-byte
// vector loads.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <type_traits>
#include <vector>

#include "tt_internal.cuh"
#include "tt_umma.cuh"

namespace tt {

// ----------------------------------------------------------- vector helpers

// (a0, a1) += w * (x0, x1) as one paired FP32 FMA (sm_100+): each lane is
// rounded exactly like fmaf, at half the issue slots.
__device__ __forceinline__ void fma2(float &a0, float &a1, float w, float x0, float x1)
{
    const float2 r = __ffma2_rn(make_float2(w, w), make_float2(x0, x1), make_float2(a0, a1));
    a0 = r.x;
    a1 = r.y;
}

template <typename T, int CPL>
__device__ __forceinline__ void fma_row(T (&acc)[CPL], T w, const T *__restrict__ p)
{
    if constexpr (sizeof(T) == 4 && CPL % 8 == 0) {
        // whole 32-byte pieces of a row (the row and the lane's chunk start
        // on 32-byte boundaries): 256-bit loads (100^3, l_max 6 adjoint, 8
        // floats per lane: 4.02 -> 3.80 ms against 16-byte loads)
#pragma unroll
        for (int t = 0; t < CPL / 8; ++t) {
            unsigned x[8];
            asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                         : "=r"(x[0]), "=r"(x[1]), "=r"(x[2]), "=r"(x[3]), "=r"(x[4]), "=r"(x[5]), "=r"(x[6]),
                           "=r"(x[7])
                         : "l"(p + 8 * t));
#pragma unroll
            for (int i = 0; i < 8; i += 2)
                fma2(acc[8 * t + i], acc[8 * t + i + 1], w, __uint_as_float(x[i]), __uint_as_float(x[i + 1]));
        }
    } else if constexpr (sizeof(T) == 4) {
        static_assert(CPL % 4 == 0, "float rows are read as float4");
#pragma unroll
        for (int t = 0; t < CPL / 4; ++t) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(p) + t);
            fma2(acc[4 * t + 0], acc[4 * t + 1], w, x.x, x.y);
            fma2(acc[4 * t + 2], acc[4 * t + 3], w, x.z, x.w);
        }
    } else {
        static_assert(CPL % 2 == 0, "double rows are read as double2");
#pragma unroll
        for (int t = 0; t < CPL / 2; ++t) {
            double2 x = __ldg(reinterpret_cast<const double2 *>(p) + t);
            acc[2 * t + 0] = fma(w, x.x, acc[2 * t + 0]);
            acc[2 * t + 1] = fma(w, x.y, acc[2 * t + 1]);
        }
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void store_row(T *__restrict__ p, const T (&v)[CPL], T scale)
{
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int t = 0; t < CPL / 4; ++t)
            reinterpret_cast<float4 *>(p)[t] =
                make_float4(scale * v[4 * t], scale * v[4 * t + 1], scale * v[4 * t + 2], scale * v[4 * t + 3]);
    } else {
#pragma unroll
        for (int t = 0; t < CPL / 2; ++t)
            reinterpret_cast<double2 *>(p)[t] = make_double2(scale * v[2 * t], scale * v[2 * t + 1]);
    }
}

// ------------------------------------------------ reduced-precision storage
// The coefficient volume may be stored as S = __nv_bfloat16 or __half while
// all arithmetic stays in T = float.  These helpers read / write CPL
// consecutive elements of a row in S.
__device__ __forceinline__ float2 unpack2(unsigned u, __nv_bfloat16 *)
{
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}
__device__ __forceinline__ float2 unpack2(unsigned u, __half *)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(&u));
}
__device__ __forceinline__ unsigned pack2(float a, float b, __nv_bfloat16 *)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned *>(&v);
}
__device__ __forceinline__ unsigned pack2(float a, float b, __half *)
{
    __half2 v = __floats2half2_rn(a, b);
    return *reinterpret_cast<unsigned *>(&v);
}

template <typename T, typename S, int CPL>
__device__ __forceinline__ void fma_row_s(T (&acc)[CPL], T w, const S *__restrict__ p)
{
    if constexpr (std::is_same<T, S>::value) {
        fma_row<T, CPL>(acc, w, p);
    } else {
        static_assert(sizeof(S) == 2 && CPL % 4 == 0, "2-byte storage rows are read 4 or 8 elements at a time");
        if constexpr (CPL % 8 == 0) {
#pragma unroll
            for (int t = 0; t < CPL / 8; ++t) {
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p) + t);
                const unsigned uu[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = unpack2(uu[k], (S *)nullptr);
                    fma2(acc[8 * t + 2 * k], acc[8 * t + 2 * k + 1], w, f.x, f.y);
                }
            }
        } else {
#pragma unroll
            for (int t = 0; t < CPL / 4; ++t) {
                const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p) + t);
                const float2 f0 = unpack2(u.x, (S *)nullptr), f1 = unpack2(u.y, (S *)nullptr);
                fma2(acc[4 * t], acc[4 * t + 1], w, f0.x, f0.y);
                fma2(acc[4 * t + 2], acc[4 * t + 3], w, f1.x, f1.y);
            }
        }
    }
}

// ----------------------------------------------------- wide row-piece loads
// NB bytes from p (aligned to ALIGN bytes) as 32-bit words, in pieces of 32
// bytes (the 256-bit global load of sm_100+) where size and alignment allow,
// else 16 or 8.  A quarter-warp whose lanes read one contiguous 128-byte run
// moves it as one L1 wavefront; lanes of four-lane groups reading separate
// 64-byte rows take about 1.45x the wavefronts for the same bytes.  SAFE:
// every address the caller can form is in bounds, even for an iteration the
// compiler executes speculatively, so the 256-bit load may be scheduled
// freely (not volatile) and loads of several planes overlap.
template <int NB, int ALIGN, bool SAFE = false>
__device__ __forceinline__ void ldg_words(const void *p, unsigned (&w)[NB / 4])
{
    constexpr int PIECE = (ALIGN >= 32 && NB % 32 == 0) ? 32 : ((ALIGN >= 16 && NB % 16 == 0) ? 16 : 8);
    static_assert(NB % PIECE == 0 && ALIGN >= 8, "row pieces are whole 8-byte words");
    const char *b = reinterpret_cast<const char *>(p);
#pragma unroll
    for (int t = 0; t < NB / PIECE; ++t) {
        if constexpr (PIECE == 32) {
            unsigned *o = w + 8 * t;
            if constexpr (SAFE)
                asm("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]), "=r"(o[7])
                    : "l"(b + 32 * t));
            else
                asm volatile("ld.global.nc.v8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                             : "=r"(o[0]), "=r"(o[1]), "=r"(o[2]), "=r"(o[3]), "=r"(o[4]), "=r"(o[5]), "=r"(o[6]),
                               "=r"(o[7])
                             : "l"(b + 32 * t));
        } else if constexpr (PIECE == 16) {
            const uint4 u = __ldg(reinterpret_cast<const uint4 *>(b + 16 * t));
            w[4 * t] = u.x; w[4 * t + 1] = u.y; w[4 * t + 2] = u.z; w[4 * t + 3] = u.w;
        } else {
            const uint2 u = __ldg(reinterpret_cast<const uint2 *>(b + 8 * t));
            w[2 * t] = u.x; w[2 * t + 1] = u.y;
        }
    }
}

// Element e of S held in the words w, converted to T.
template <typename T, typename S, int NW>
__device__ __forceinline__ T word_elem(const unsigned (&w)[NW], int e)
{
    if constexpr (std::is_same<S, float>::value) {
        return __uint_as_float(w[e]);
    } else if constexpr (std::is_same<S, double>::value) {
        return __hiloint2double((int)w[2 * e + 1], (int)w[2 * e]);
    } else {
        const float2 f = unpack2(w[e / 2], (S *)nullptr);
        return (e & 1) ? f.y : f.x;
    }
}

// acc[i] += wt * x[OFS + i] for i < N, x the NE elements of S held in w;
// paired FP32 FMAs for float.
template <typename T, typename S, int N, int OFS, int NW>
__device__ __forceinline__ void fma_words(T (&acc)[N], T wt, const unsigned (&w)[NW])
{
    if constexpr (std::is_same<T, float>::value) {
        static_assert(N % 2 == 0 && OFS % 2 == 0, "paired FMAs");
#pragma unroll
        for (int i = 0; i < N; i += 2)
            fma2(acc[i], acc[i + 1], wt, word_elem<T, S>(w, OFS + i), word_elem<T, S>(w, OFS + i + 1));
    } else {
#pragma unroll
        for (int i = 0; i < N; ++i) acc[i] = fma(wt, word_elem<T, S>(w, OFS + i), acc[i]);
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// Deterministic block sum (fixed order) of one double per thread; result in
// thread 0.
__device__ __forceinline__ double block_sum(double v, double *red)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// Sum of p[0..n) in a fixed order, for a block of kThreads threads: thread t
// keeps eight running sums over t + kThreads i (i = 0, 1, ... taken round
// robin), adds them pairwise, then block_sum.  The eight independent load
// chains keep a single-CTA reduction short.  The result is valid on thread 0.
__device__ __forceinline__ double sum_fixed_order(const double *__restrict__ p, long long n, double *red)
{
    constexpr long long B = kThreads;
    double v8[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    long long t = threadIdx.x;
    for (; t + 7 * B < n; t += 8 * B) {
#pragma unroll
        for (int i = 0; i < 8; ++i) v8[i] += __ldg(p + t + i * B);
    }
#pragma unroll
    for (int i = 0; i < 7; ++i)
        if (t + i * B < n) v8[i] += __ldg(p + t + i * B);
    const double v = ((v8[0] + v8[1]) + (v8[2] + v8[3])) + ((v8[4] + v8[5]) + (v8[6] + v8[7]));
    return block_sum(v, red);
}

// Transverse coordinates of ray (j, k) on plane 0, u0 + j uj + k uk and
// v0 + j vj + k vk, in FP64 with explicit FMAs (one rounding order for every
// kernel that marches rays), rounded once to T.
template <typename T>
__device__ __forceinline__ void ray_base(const ProjGeom &P, int j, int k, T &ur, T &vr)
{
    ur = (T)__fma_rn((double)k, P.uk, __fma_rn((double)j, P.uj, P.u0));
    vr = (T)__fma_rn((double)k, P.vk, __fma_rn((double)j, P.vj, P.v0));
}

// Range of planes p in [0, Nm-1] on which coordinate w(p) = w0 + p*dw lies
// in (-1, N), i.e. can give a bilinear tap inside [0, N-1].  floor/ceil of the
// bounds may add one plane on each side; those planes see only the zero
// border of the padded volume.
template <typename T>
__device__ __forceinline__ void clip_planes(T w0, T dw, int N, T &lo, T &hi)
{
    if (fabs(dw) < T(1e-12)) {
        if (!(w0 > T(-1) && w0 < T(N))) { lo = T(1); hi = T(0); }
        return;
    }
    T inv = T(1) / dw;
    T p1 = (T(-1) - w0) * inv, p2 = (T(N) - w0) * inv;
    lo = fmax(lo, fmin(p1, p2));
    hi = fmin(hi, fmax(p1, p2));
}

// SH contraction of a marched ray and, in GRAD mode, the residual, its
// weighted square and the back-contraction (Eq. forward_model, Eq. residual).
// The contraction runs four segments at a time: partial dot products over the
// lane's CPL channels (chunk `chunk` of the row), a butterfly across the LG
// lanes of the channel group, then each lane back-contracts into its own
// channels.  Lanes with
// writer == false (duplicate halves) compute but do not store.  Returns the
// ray's sum of W r^2 on every lane.
template <typename T, typename S, int CPL, int KP, int LG, bool GRAD>
__device__ __forceinline__ T forward_epilogue(const T (&acc)[CPL], int q, int chunk, bool valid, bool writer,
                                              long long pix,
                                              const T *__restrict__ Bs, int C, int CP, T *__restrict__ Iout,
                                              const T *__restrict__ Id, const T *__restrict__ Wd,
                                              T *__restrict__ G)
{
    T gacc[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) gacc[i] = T(0);
    T lossr = T(0);
    const int boff = chunk * CPL;
    const bool vec4 = (C % 4) == 0;
    for (int c0 = 0; c0 < CP; c0 += 4) {
        T ih[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const T *brow = Bs + (c0 + t) * KP + boff;
            T sacc = T(0);
#pragma unroll
            for (int i = 0; i < CPL; ++i) sacc = fma(brow[i], acc[i], sacc);
            ih[t] = sacc;
        }
#pragma unroll
        for (int off = LG / 2; off > 0; off >>= 1)
#pragma unroll
            for (int t = 0; t < 4; ++t) ih[t] += __shfl_xor_sync(0xffffffffu, ih[t], off);
        if constexpr (!GRAD) {
            if (valid && writer) {
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if ((t % LG) == q && c0 + t < C) Iout[pix * C + c0 + t] = ih[t];
            }
        } else {
            T dI[4] = {T(0), T(0), T(0), T(0)}, dW[4] = {T(1), T(1), T(1), T(1)};
            if (valid) {
                const long long o = pix * C + c0;
                if (vec4) {
                    if constexpr (sizeof(T) == 4) {
                        float4 a = __ldg(reinterpret_cast<const float4 *>(Id + o));
                        dI[0] = a.x; dI[1] = a.y; dI[2] = a.z; dI[3] = a.w;
                        if (Wd) {
                            float4 b = __ldg(reinterpret_cast<const float4 *>(Wd + o));
                            dW[0] = b.x; dW[1] = b.y; dW[2] = b.z; dW[3] = b.w;
                        }
                    } else {
                        double2 a0 = __ldg(reinterpret_cast<const double2 *>(Id + o));
                        double2 a1 = __ldg(reinterpret_cast<const double2 *>(Id + o) + 1);
                        dI[0] = a0.x; dI[1] = a0.y; dI[2] = a1.x; dI[3] = a1.y;
                        if (Wd) {
                            double2 b0 = __ldg(reinterpret_cast<const double2 *>(Wd + o));
                            double2 b1 = __ldg(reinterpret_cast<const double2 *>(Wd + o) + 1);
                            dW[0] = b0.x; dW[1] = b0.y; dW[2] = b1.x; dW[3] = b1.y;
                        }
                    }
                } else {
#pragma unroll
                    for (int t = 0; t < 4; ++t)
                        if (c0 + t < C) {
                            dI[t] = __ldg(Id + o + t);
                            if (Wd) dW[t] = __ldg(Wd + o + t);
                        }
                }
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const bool live = valid && (c0 + t < C);
                const T rr = live ? ih[t] - dI[t] : T(0);
                const T wr = live ? dW[t] * rr : T(0);
                lossr = fma(wr, rr, lossr);
                const T *brow = Bs + (c0 + t) * KP + boff;
#pragma unroll
                for (int i = 0; i < CPL; ++i) gacc[i] = fma(brow[i], wr, gacc[i]);
            }
        }
    }
    if constexpr (GRAD) {
        if (valid && writer) store_row<T, CPL>(G + pix * KP + chunk * CPL, gacc, T(2));
    }
    return lossr;
}

// ------------------------------------------------------------ forward kernel
//
// One CTA = one projection s x one 8-wide tile of rays.  Each lane group
// marches its ray along the main axis (Joseph's method, bilinear taps read
// straight from the L1/L2-resident volume), scales by the step length, then
//   PROJECT: writes I_hat = B_s Y                           (Eq. forward_model)
//   GRAD:    r = I_hat - I, loss += W r^2, G = 2 B_s^T (W r) (Eq. residual)
// The SH contraction runs four segments at a time: partial dot products over
// the lane's channels, a butterfly across the lane group, then each lane
// back-contracts into its own channels.
template <typename T, typename S, int KP, int LG, bool GRAD>
__global__ void __launch_bounds__(kFwdThreads)
k_forward(const ProjGeom *__restrict__ geo, const S *__restrict__ cpad /* interior origin */,
          const S *__restrict__ cpadx /* interior origin of the x-innermost copy, or NULL */, const T *__restrict__ Bp,
          int nj, int nk, int C, int CP, int tiles_k, int slab_order, int s_base,
          T *__restrict__ Iout, const T *__restrict__ Id, const T *__restrict__ Wd,
          T *__restrict__ G, double *__restrict__ partials)
{
    constexpr int CPL = KP / LG;
    constexpr int TK = fwd_tk(LG);
    constexpr int TJ = fwd_tj(LG);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Bs = reinterpret_cast<T *>(smem_raw);   // [CP][KP]
    __shared__ double red[kFwdThreads / 32];

    // CTA order.  slab_order == 0: all tiles of one projection, projection by
    // projection (gridDim = (tiles_k * tiles_j, S)).  slab_order == 1: k tile
    // fastest, then projection, then j tile (gridDim = (tiles_k * S, tiles_j)),
    // so that the CTAs in flight march the same few detector rows of many
    // projections -- for rotations about the j axis the same y-slab of the
    // volume, which then stays in L2 when the whole volume does not fit.
    // The launch covers projections s_base, s_base + 1, ... (all of them, or
    // one chunk of a pipelined host-buffer evaluation).
    int tk, s, tj, tiles_j;
    if (slab_order) { tk = blockIdx.x % tiles_k; s = s_base + blockIdx.x / tiles_k; tj = blockIdx.y; tiles_j = gridDim.y; }
    else { s = s_base + blockIdx.y; tj = blockIdx.x / tiles_k; tk = blockIdx.x % tiles_k; tiles_j = gridDim.x / tiles_k; }
    const int r = threadIdx.x / LG, q = threadIdx.x % LG;
    const int j = tj * TJ + r / TK, k = tk * TK + r % TK;
    const bool valid = (j < nj) && (k < nk);

    const T *Bsrc = Bp + (size_t)s * CP * KP;
    for (int t = threadIdx.x; t < CP * KP; t += kFwdThreads) Bs[t] = Bsrc[t];

    const ProjGeom &P = geo[s];
    // Ray base in FP64 (one rounding to T), per-plane stepping in T.
    T ur, vr;
    ray_base<T>(P, j, k, ur, vr);
    const T up = (T)P.up, vp = (T)P.vp;
    const int Nu = P.Nu, Nv = P.Nv, sm = P.sm, su = P.su;
    T lo = T(0), hi = T(P.Nm - 1);
    clip_planes<T>(ur, up, Nu, lo, hi);
    clip_planes<T>(vr, vp, Nv, lo, hi);
    int plo = valid ? max(0, (int)floor(lo)) : 1;
    int phi = valid ? min(P.Nm - 1, (int)ceil(hi)) : 0;
    if (cpad == nullptr) phi = plo - 1;   // a zero volume: every ray sum is exactly zero, nothing to march

    // The march reads bilinear taps in pairs along v, the innermost axis of
    // the volume copy this projection reads (sv == 1): rows (iu, iv) and
    // (iu, iv + 1) are one contiguous piece of 2 KP elements, and likewise
    // at iu + 1.  Lane q of the group reads part q of each pair, NP = 2 KP /
    // LG elements: for LG >= 2 that is row iv + h, h = q / (LG / 2), channels
    // [cofs, cofs + NP); a lone lane (LG == 1) reads both rows.  Lanes h = 0
    // and h = 1 sum their halves once the ray is marched.
    constexpr int NP = 2 * KP / LG;
    constexpr int ACH = LG == 1 ? KP : NP;          // channels a lane accumulates
    constexpr int ROWB = KP * (int)sizeof(S);
    constexpr int PIECEB = NP * (int)sizeof(S);
    constexpr int ALIGN = LG == 1 ? (ROWB & -ROWB) : ((ROWB | PIECEB) & -(ROWB | PIECEB));
    constexpr int NW = PIECEB / 4;
    const int h = LG == 1 ? 0 : q / (LG / 2);
    const int cofs = LG == 1 ? 0 : (q % (LG / 2)) * NP;
    T acc[ACH];
#pragma unroll
    for (int i = 0; i < ACH; ++i) acc[i] = T(0);
    // cpad is the interior origin of a volume with a two-voxel zero border:
    // every tap index in [-2, N+1] is a valid address, so the loads need no
    // bounds tests (indices are clamped to [-2, N] first, which only ever
    // moves a tap pair that lies wholly in the border).
    const S *cq = (P.copy ? cpadx : cpad) + q * NP;
    const long long sub = (long long)su * KP;
    // Reduced-precision storage (S = bf16 / f16) is read and converted per
    // tap; the ray sum stays a plain FP32 accumulation: over N planes its
    // rounding (~N 2^-24) is far below the 2^-9 / 2^-12 rounding of the
    // stored values (compensated sums were measured to change the projection
    // by < 1e-9 relative, at 10% of the kernel's time).
    // Loads in flight per lane: 32-channel rows march two planes per
    // iteration and 2-byte rows of up to 16 channels four (measured at 64^3:
    // bfloat16 0.313 -> 0.277 ms); FP32 rows of 16 channels hold 16 words
    // per plane already, and unrolling them was measured slower.
    constexpr int kUnroll = KP == 32 ? 2 : ((sizeof(S) == 2 && KP <= 16) ? 4 : 1);
#pragma unroll kUnroll
    for (int p = plo; p <= phi; ++p) {
        const T u = fma((T)p, up, ur), v = fma((T)p, vp, vr);
        const T fu = floor(u), fv = floor(v);
        const int iu = min(max((int)fu, -2), Nu), iv = min(max((int)fv, -2), Nv);
        const T wu = u - fu, wv = v - fv;
        const S *t0 = cq + ((long long)p * sm + (long long)iu * su + iv) * KP;
        unsigned x0[NW], x1[NW];
        // any p in [plo - 1, phi + 1] and the clamped iu, iv address the padded
        // volume (two-voxel border), so the loads may run speculatively
        ldg_words<PIECEB, ALIGN, true>(t0, x0);
        ldg_words<PIECEB, ALIGN, true>(t0 + sub, x1);
        if constexpr (LG >= 2) {
            const T wvh = h ? wv : T(1) - wv;
            fma_words<T, S, ACH, 0>(acc, (T(1) - wu) * wvh, x0);
            fma_words<T, S, ACH, 0>(acc, wu * wvh, x1);
        } else {
            const T a0 = T(1) - wu, b0 = T(1) - wv;
            fma_words<T, S, ACH, 0>(acc, a0 * b0, x0);
            fma_words<T, S, ACH, KP>(acc, a0 * wv, x0);
            fma_words<T, S, ACH, 0>(acc, wu * b0, x1);
            fma_words<T, S, ACH, KP>(acc, wu * wv, x1);
        }
    }
    // Both rows' sums in every lane of a pair, then lane q keeps channel
    // chunk `chunk` (CPL channels) for the epilogue.
    T accq[CPL];
    int chunk = 0;
    if constexpr (LG >= 2) {
#pragma unroll
        for (int i = 0; i < ACH; ++i) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], LG / 2);
#pragma unroll
        for (int i = 0; i < CPL; ++i) accq[i] = h ? acc[CPL + i] : acc[i];
        chunk = cofs / CPL + h;
    } else {
#pragma unroll
        for (int i = 0; i < CPL; ++i) accq[i] = acc[i];
    }
    const T step = (T)P.step;
#pragma unroll
    for (int i = 0; i < CPL; ++i) accq[i] *= step;

    __syncthreads();   // Bs staged

    const long long pix = ((long long)s * nj + j) * nk + k;
    const T lossr = forward_epilogue<T, S, CPL, KP, LG, GRAD>(accq, q, chunk, valid, true, pix, Bs, C, CP, Iout, Id,
                                                              Wd, G);
    if constexpr (GRAD) {
        double tot;
        if constexpr (std::is_same<T, float>::value)
            tot = dot2_block_sum(Dot2{(q == 0 && valid) ? lossr : 0.f, 0.f}, reinterpret_cast<Dot2 *>(red));
        else
            tot = block_sum((q == 0 && valid) ? (double)lossr : 0.0, red);
        // canonical CTA index (projection, j tile, k tile): the same for
        // either CTA order and for chunked launches, so the loss sums alike
        if (threadIdx.x == 0) partials[((long long)s * tiles_j + tj) * tiles_k + tk] = tot;
    }
}

// --------------------------------------------- staged forward (FP32, KP = 16)
//
// The ray sums of k_forward with the bilinear taps read from shared memory.
// One CTA = one projection x a tile of kStTJ x kStTK rays.  Warp 8 (the copy
// warp) walks the tile's planes and, for each, copies the box of the padded
// volume copy that holds the tile's taps -- st_ru rows along u of st_rv
// voxels along v, one plane thick -- into the next stage of a ring with one
// tiled tensor copy, completing on the stage's `full` mbarrier; a stage is
// refilled once all eight consumer warps have arrived on its `empty`
// mbarrier.  Parallel rays shift rigidly from plane to plane, so the box of an
// 8 x 16 tile holds about half as many voxels as the tile reads taps, and
// every read hits shared memory.  The ring has room for kStRing boxes of the
// largest size over the projections; a projection whose boxes are smaller
// runs min(kStMaxDepth, room / box) stages, so more planes are in flight.
// (One tensor copy per plane: bulk copies of the box's rows one by one were
// measured to cost a request each, three times the time of the bytes.)
//
// Consumers: four lanes per ray and two rays per lane group (j and j + 4).
// Lane q owns the eight floats [8q, 8q + 8) of each tap pair, exactly as in
// k_forward, read as two 16-byte chunks 2q and 2q + 1; lanes of odd groups
// read them in the order (2q + 1, 2q).  A quarter-warp (two groups) then
// reads, per instruction, the even chunks of one pair and the odd chunks of
// the other, whose 16-byte bank groups differ for any two pairs that start on
// 64-byte boundaries: no bank conflicts.  Per plane each ray adds the pair of
// row iu, then that of row iu + 1, with k_forward's weights in k_forward's
// order, so both kernels give the same FP32 sums bit for bit.
//
// A wait that gives up (a bounded number of polls) makes the tile's rays
// NaN, which the loss and every output show; the copy warp waits (bounded)
// for its copies in flight before the CTA exits.
struct StageHdr {
    int ulo, vlo;
};
constexpr uint32_t kStWaitTries = 1u << 22;

// First row of a box of n rows that holds floor(c) and floor(c) + 1 for every
// coordinate c in [cmin, cmax], the start clamped to [-2, N] (where the
// clamped tap indices of k_forward lie).
__device__ __forceinline__ int stage_lo(float cmin, int N)
{
    return min(max((int)floorf(cmin - kStEps), -2), N);
}

template <bool GRAD>
__global__ void __launch_bounds__(kStThreads, 2)
k_forward_staged(const ProjGeom *__restrict__ geo, const TmaDesc *__restrict__ tmaps, const float *__restrict__ Bp,
                 int nj, int nk, int C, int CP, int tiles_k, int slab_order, int s_base, int cap,
                 float *__restrict__ Iout, const float *__restrict__ Id, const float *__restrict__ Wd,
                 float *__restrict__ G, double *__restrict__ partials)
{
    constexpr int KP = 16, LG = 4, CPL = 4, NR = 2;
    // The tensor copies write 128-byte aligned stages: the dynamic shared
    // memory holds 128 bytes of slack and the ring starts at its first
    // 128-byte boundary.
    extern __shared__ __align__(1024) unsigned char st_smem[];
    unsigned char *ring = st_smem + ((128u - (umma::smem_u32(st_smem) & 127u)) & 127u);
    float *stages = reinterpret_cast<float *>(ring);           // kStRing * cap voxels of KP floats
    float *Bs = stages + (size_t)kStRing * cap * KP;           // [CP][KP]
    __shared__ __align__(8) uint64_t full[kStMaxDepth], empty[kStMaxDepth];
    __shared__ StageHdr hdr[kStMaxDepth];
    __shared__ int prange[2];
    __shared__ Dot2 red[kStThreads / 32];

    int tk, s, tj, tiles_j;
    if (slab_order) { tk = blockIdx.x % tiles_k; s = s_base + blockIdx.x / tiles_k; tj = blockIdx.y; tiles_j = gridDim.y; }
    else { s = s_base + blockIdx.y; tj = blockIdx.x / tiles_k; tk = blockIdx.x % tiles_k; tiles_j = gridDim.x / tiles_k; }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool copier = warp == kStConsumers / 32;

    const float *Bsrc = Bp + (size_t)s * CP * KP;
    for (int t = threadIdx.x; t < CP * KP; t += kStThreads) Bs[t] = Bsrc[t];
    if (threadIdx.x == 0) {
        for (int i = 0; i < kStMaxDepth; ++i) {
            umma::mbar_init(&full[i], 1);
            umma::mbar_init(&empty[i], kStConsumers / 32);
        }
        prange[0] = INT_MAX;
        prange[1] = INT_MIN;
    }
    __syncthreads();

    const ProjGeom &P = geo[s];
    const float up = (float)P.up, vp = (float)P.vp;
    const int Nu = P.Nu, Nv = P.Nv;

    // consumer rays: group g, lane q; rays (j0 + 4 r, k)
    const int g = threadIdx.x / LG, q = threadIdx.x % LG;
    const int k = tk * kStTK + g % kStTK, j0 = tj * kStTJ + g / kStTK;
    float ur[NR], vr[NR];
    int plo[NR], phi[NR];
    bool valid[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int j = j0 + 4 * r;
        valid[r] = !copier && j < nj && k < nk;
        ray_base<float>(P, j, k, ur[r], vr[r]);
        float lo = 0.f, hi = (float)(P.Nm - 1);
        clip_planes<float>(ur[r], up, Nu, lo, hi);
        clip_planes<float>(vr[r], vp, Nv, lo, hi);
        plo[r] = valid[r] ? max(0, (int)floorf(lo)) : 1;
        phi[r] = valid[r] ? min(P.Nm - 1, (int)ceilf(hi)) : 0;
        if (q == 0 && plo[r] <= phi[r]) {
            atomicMin(&prange[0], plo[r]);
            atomicMax(&prange[1], phi[r]);
        }
    }
    __syncthreads();
    const int p0 = prange[0], np = prange[1] >= prange[0] ? prange[1] - prange[0] + 1 : 0;

    float acc[NR][8];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int i = 0; i < 8; ++i) acc[r][i] = 0.f;
    bool ok = true;

    // This projection's ring: stages of ru x rv voxels, rounded up to an even
    // count so that every stage starts on a 128-byte boundary.
    const int ru = P.st_ru, rv = P.st_rv;
    const int sstride = (ru * rv + 1) & ~1;
    const int depth = min(kStMaxDepth, (kStRing * cap) / sstride);

    if (copier) {
        // Lower tile extents at plane 0 from its corner rays (the coordinates
        // are affine in j, k; the corners are those of the rays inside the
        // detector), computed like each ray's.
        const int jc = min(tj * kStTJ + ((lane & 1) ? kStTJ - 1 : 0), nj - 1);
        const int kc = min(tk * kStTK + ((lane & 2) ? kStTK - 1 : 0), nk - 1);
        float umin, vmin;
        ray_base<float>(P, jc, kc, umin, vmin);
#pragma unroll
        for (int off = 1; off <= 2; off <<= 1) {
            umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, off));
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
        }
        if (lane == 0) {   // one thread issues every copy of the tile
            const TmaDesc *tm = tmaps + s;
            umma::tensormap_acquire(tm);
            int st = 0, ph = 0, issued = 0;
            for (int n = 0; n < np; ++n) {
                if (n >= depth && !umma::mbar_wait(&empty[st], ph ^ 1, kStWaitTries)) break;
                const float pf = (float)(p0 + n);
                const int ulo = stage_lo(fmaf(pf, up, umin), Nu), vlo = stage_lo(fmaf(pf, vp, vmin), Nv);
                hdr[st] = StageHdr{ulo, vlo};
                umma::mbar_arrive_expect_tx(&full[st], (uint32_t)(ru * rv * KP * 4));
                // tensor coordinates of the padded copy: voxel index + 2, 8 words per voxel
                const int pc = p0 + n + 2, uc = ulo + 2;
                umma::tma_load_3d(stages + (size_t)st * sstride * KP, tm, 8 * (vlo + 2), P.st_umid ? uc : pc,
                                  P.st_umid ? pc : uc, &full[st]);
                issued = n + 1;
                if (++st == depth) { st = 0; ph ^= 1; }
            }
            // no copy may still be writing shared memory when the CTA exits
            for (int n = max(0, issued - depth); n < issued; ++n)
                umma::mbar_wait(&full[n % depth], (n / depth) & 1, kStWaitTries);
        }
        __syncwarp();
    } else {
        const int pi = g & 1;
        const int c0 = 2 * q + pi, c1 = 2 * q + 1 - pi;   // 16-byte chunks of a pair, in read order
        const int h = q >> 1;                             // voxel iv + h of the pair holds lane q's channels
        const int lim = ru * rv - rv - 2;                 // keeps both pairs of a tap inside the box
        int st = 0, ph = 0;
        for (int n = 0; n < np; ++n) {
            // every lane observes the stage's completion; the warp gives up as one
            if (!__all_sync(0xffffffffu, umma::mbar_wait(&full[st], ph, kStWaitTries))) { ok = false; break; }
            const StageHdr hd = hdr[st];
            const float *sb = stages + (size_t)st * sstride * KP;
            const int p = p0 + n;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                if (p < plo[r] || p > phi[r]) continue;
                const float u = fmaf((float)p, up, ur[r]), v = fmaf((float)p, vp, vr[r]);
                const float fu = floorf(u), fv = floorf(v);
                const int iu = min(max((int)fu, -2), Nu), iv = min(max((int)fv, -2), Nv);
                const float wu = u - fu, wv = v - fv;
                const int idx = min(max((iu - hd.ulo) * rv + (iv - hd.vlo), 0), lim);
                const float *t0 = sb + (size_t)idx * KP;
                const float *t1 = t0 + (size_t)rv * KP;
                const float4 a0 = *reinterpret_cast<const float4 *>(t0 + 4 * c0);
                const float4 a1 = *reinterpret_cast<const float4 *>(t0 + 4 * c1);
                const float4 b0 = *reinterpret_cast<const float4 *>(t1 + 4 * c0);
                const float4 b1 = *reinterpret_cast<const float4 *>(t1 + 4 * c1);
                const float wvh = h ? wv : 1.f - wv;
                const float w0 = (1.f - wu) * wvh, w1 = wu * wvh;
                float *A = acc[r];
                fma2(A[0], A[1], w0, a0.x, a0.y);
                fma2(A[2], A[3], w0, a0.z, a0.w);
                fma2(A[4], A[5], w0, a1.x, a1.y);
                fma2(A[6], A[7], w0, a1.z, a1.w);
                fma2(A[0], A[1], w1, b0.x, b0.y);
                fma2(A[2], A[3], w1, b0.z, b0.w);
                fma2(A[4], A[5], w1, b1.x, b1.y);
                fma2(A[6], A[7], w1, b1.z, b1.w);
            }
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&empty[st]);
            if (++st == depth) { st = 0; ph ^= 1; }
        }
        if (pi) {   // chunk order back to (2q, 2q + 1)
#pragma unroll
            for (int r = 0; r < NR; ++r)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float t = acc[r][i];
                    acc[r][i] = acc[r][4 + i];
                    acc[r][4 + i] = t;
                }
        }
    }
    __syncthreads();

    Dot2 lossr{0.f, 0.f};
    if (!copier) {
        const float step = (float)P.step;
        const int chunk = (q % 2) * 2 + (q >> 1);
        const float bad = __int_as_float(0x7fc00000);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            // both voxels' sums in every lane of a pair; lane q keeps chunk `chunk`
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[r][i] += __shfl_xor_sync(0xffffffffu, acc[r][i], LG / 2);
            float accq[CPL];
#pragma unroll
            for (int i = 0; i < CPL; ++i) accq[i] = ok ? ((q >> 1) ? acc[r][CPL + i] : acc[r][i]) * step : bad;
            const long long pix = ((long long)s * nj + (j0 + 4 * r)) * nk + k;
            const float lr = forward_epilogue<float, float, CPL, KP, LG, GRAD>(accq, q, chunk, valid[r], true, pix, Bs,
                                                                           C, CP, Iout, Id, Wd, G);
            if (q == 0 && valid[r]) dot2_add1(lossr, lr);
        }
    }
    if constexpr (GRAD) {
        const double tot = dot2_block_sum(lossr, red);
        if (threadIdx.x == 0) partials[((long long)s * tiles_j + tj) * tiles_k + tk] = tot;
    }
}

// ----------------------------------------------------- back-contraction
// G[pix][i] = sum_c B[s][c][i] R[pix][c]  (the SH part of A^T).
template <typename T, typename S, int KP, int LG>
__global__ void __launch_bounds__(kThreads)
k_backcontract(const T *__restrict__ Bp, const T *__restrict__ R, T *__restrict__ G,
               long long npix, int njk, int C, int CP)
{
    constexpr int CPL = KP / LG;
    constexpr int RAYS = kThreads / LG;
    const int r = threadIdx.x / LG, q = threadIdx.x % LG;
    const long long pix = (long long)blockIdx.x * RAYS + r;
    if (pix >= npix) return;
    const int s = (int)(pix / njk);
    const T *B = Bp + (size_t)s * CP * KP + q * CPL;
    T acc[CPL];
#pragma unroll
    for (int i = 0; i < CPL; ++i) acc[i] = T(0);
    for (int c = 0; c < C; ++c) {
        const T rc = __ldg(R + pix * C + c);
#pragma unroll
        for (int i = 0; i < CPL; ++i) acc[i] = fma(__ldg(B + c * KP + i), rc, acc[i]);
    }
    store_row<T, CPL>(G + pix * KP + q * CPL, acc, T(1));
}

__device__ __forceinline__ int sel3(int x, int y, int z, int axis)
{
    return axis == 0 ? x : (axis == 1 ? y : z);
}

// ---------------------------------------------------------- adjoint kernel
//
// Exact transpose of k_forward's Joseph discretisation, as a gather (every
// voxel written once, no atomics).  On the voxel's plane of projection s, the
// rays that have voxel (U,V) as a bilinear tap are those with |u - U| < 1 and
// |v - V| < 1; each contributes its G row with weight (1-|du|)(1-|dv|) *
// step, the weight the forward gave that tap.  Those rays are the detector
// points inside a parallelogram.  They are enumerated column by column along
// one detector axis (the outer axis o; the inner axis i is the other one):
// the NO columns o0 = floor(oc - ho) + 1, ... that meet the parallelogram,
// and in column o the NI points from the first one above the column's lower
// edge, floor(ic + max(au + lu (o - oc), av + lv (o - oc))) + 1.  Per
// projection the host picks the axis order that gives fewer candidates
// (NO * NI, about 4.3 per voxel on the tilted-series workloads against 5.7
// for the bounding box) and the kernel unrolls the loop per (NO, NI).  A
// point whose true weight is positive but within FP rounding of zero may be
// left out: its contribution is below the rounding of the others.
//
// Work split: a lane group of LG lanes owns V <= LG voxels (adjacent in
// x).  Lane q does the candidate geometry for voxel q % V only, then the
// group exchanges each candidate's weight and each column's first row --
// through shared memory for FP32 (one 16-byte read gives a candidate's
// weights for all sources; shuffles would take a load-store-unit wavefront
// per source), with shuffles otherwise -- and every lane accumulates its own
// channel chunk q of that row for all V voxels (with V == 1 every lane
// already holds them).  The geometry is thus computed once per voxel while a
// G row is still read as one contiguous KP-float segment by the LG lanes
// together.  Per-projection constants travel in the kernel's parameter space.

// Candidate geometry of one voxel: weight of candidate (a, b) and first row
// of column a.  o0: first column; no, ni: detector extents along the outer
// and inner axes; so, si: their strides in rows of G.
template <typename T>
struct AdjVoxel {
    T oc, ic, bu, bv;
    int o0;
    bool valid;
};

template <typename T, int NO, int NI>
__device__ __forceinline__ void adj_geometry(const AdjVoxel<T> &vx, const AdjProj<T> &c, int n_o, int n_i, int so,
                                             int si, T (&w)[NO * NI], int (&r)[NO])
{
#pragma unroll
    for (int a = 0; a < NO; ++a) {
        const int o = vx.o0 + a;
        const T d = (T)o - vx.oc;
        const T lo = fmax(c.au + c.lu * d, c.av + c.lv * d);
        const T fi = floor(vx.ic + lo) + T(1);
        const int i0 = (int)fi;
        r[a] = i0 * si + o * so;
        const T du0 = vx.bu + (T)o * c.uo + fi * c.ui;
        const T dv0 = vx.bv + (T)o * c.vo + fi * c.vi;
        const bool col_in = vx.valid && (unsigned)o < (unsigned)n_o;
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const T du = du0 + (T)b * c.ui;
            const T dv = dv0 + (T)b * c.vi;
            const T tu = T(1) - fabs(du);
            const T tv = c.step - c.step * fabs(dv);
            const bool hit = col_in && (unsigned)(i0 + b) < (unsigned)n_i && tu > T(0) && tv > T(0);
            w[a * NI + b] = hit ? tu * tv : T(0);
        }
    }
}

// Candidates of a (NO, NI) window, exchanged by shuffles.
template <typename T, typename S, int CPL, int KP, int LG, int V, int NO, int NI>
__device__ __forceinline__ void adj_window(T (&acc)[V][CPL], const S *__restrict__ Gq, const AdjVoxel<T> &vx,
                                           const AdjProj<T> &c, int n_o, int n_i, int so, int si)
{
    T w[NO * NI];
    int r[NO];
    adj_geometry<T, NO, NI>(vx, c, n_o, n_i, so, si, w, r);
#pragma unroll
    for (int a = 0; a < NO; ++a) {
        int rs[V];
#pragma unroll
        for (int src = 0; src < V; ++src) rs[src] = (LG == 1 || V == 1) ? r[a] : __shfl_sync(0xffffffffu, r[a], src, LG);
#pragma unroll
        for (int b = 0; b < NI; ++b) {
#pragma unroll
            for (int src = 0; src < V; ++src) {
                const T ws = (LG == 1 || V == 1) ? w[a * NI + b] : __shfl_sync(0xffffffffu, w[a * NI + b], src, LG);
                if (ws != T(0)) fma_row_s<T, S, CPL>(acc[src], ws, Gq + (long long)(rs[src] + b * si) * KP);
            }
        }
    }
}

// Same, exchanged through shared memory: lane q publishes its voxel's
// weights (one store per candidate) and column rows, then every lane reads
// the V sources' weights of a candidate with one 16-byte load.
template <typename S, int CPL, int KP, int LG, int V, int NO, int NI>
__device__ __forceinline__ void adj_window_sm(float (&acc)[V][CPL], const S *__restrict__ Gq,
                                              const AdjVoxel<float> &vx, const AdjProj<float> &c, int n_o, int n_i,
                                              int so, int si, float *__restrict__ wb, int *__restrict__ rb, int q)
{
    static_assert(V >= 2 && V <= 4 && NO <= 3 && NO * NI <= 9, "exchange holds 4 sources x 9 candidates, 3 columns");
    float w[NO * NI];
    int r[NO];
    adj_geometry<float, NO, NI>(vx, c, n_o, n_i, so, si, w, r);
    if (q < V) {
#pragma unroll
        for (int a = 0; a < NO; ++a) rb[a * 4 + q] = r[a];
#pragma unroll
        for (int t = 0; t < NO * NI; ++t) wb[t * 4 + q] = w[t];
    }
    __syncwarp();
#pragma unroll
    for (int a = 0; a < NO; ++a) {
        const int4 r4 = *reinterpret_cast<const int4 *>(rb + a * 4);
        const int rs[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
        for (int b = 0; b < NI; ++b) {
            const float4 w4 = *reinterpret_cast<const float4 *>(wb + (a * NI + b) * 4);
            const float ws[4] = {w4.x, w4.y, w4.z, w4.w};
            // Rows of 12 or more floats per lane: predicated load and
            // unconditional FMAs (a zero weight adds exactly zero, the skipped
            // row reads as zeros) instead of a branch per source -- measured
            // 14.62 -> 14.27 ms for the l_max 8 adjoint at 128^3, but slower
            // for 4 and 8 floats per lane (64^3: 0.366 -> 0.394 ms).
            constexpr bool kPred = CPL >= 12 && std::is_same<S, float>::value;
#pragma unroll
            for (int src = 0; src < V; ++src) {
                if constexpr (kPred) {
                    float x[CPL];
#pragma unroll
                    for (int i = 0; i < CPL; ++i) x[i] = 0.f;
                    if (ws[src] != 0.f) {
                        const float4 *p4 = reinterpret_cast<const float4 *>(Gq + (long long)(rs[src] + b * si) * KP);
#pragma unroll
                        for (int t = 0; t < CPL / 4; ++t) {
                            const float4 v = __ldg(p4 + t);
                            x[4 * t] = v.x; x[4 * t + 1] = v.y; x[4 * t + 2] = v.z; x[4 * t + 3] = v.w;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < CPL; i += 2) fma2(acc[src][i], acc[src][i + 1], ws[src], x[i], x[i + 1]);
                } else if (ws[src] != 0.f) {
                    fma_row_s<float, S, CPL>(acc[src], ws[src], Gq + (long long)(rs[src] + b * si) * KP);
                }
            }
        }
    }
    __syncwarp();
}

// Any window size (geometries with strongly unequal voxel and pixel sizes):
// runtime loops, shuffles.
template <typename T, typename S, int CPL, int KP, int LG, int V>
__device__ __forceinline__ void adj_window_any(T (&acc)[V][CPL], const S *__restrict__ Gq, const AdjVoxel<T> &vx,
                                               const AdjProj<T> &c, int n_o, int n_i, int so, int si, int NO, int NI)
{
    for (int a = 0; a < NO; ++a) {
        const int o = vx.o0 + a;
        const T d = (T)o - vx.oc;
        const T lo = fmax(c.au + c.lu * d, c.av + c.lv * d);
        const T fi = floor(vx.ic + lo) + T(1);
        const int i0 = (int)fi;
        const int r = i0 * si + o * so;
        const T du0 = vx.bu + (T)o * c.uo + fi * c.ui;
        const T dv0 = vx.bv + (T)o * c.vo + fi * c.vi;
        for (int b = 0; b < NI; ++b) {
            const T du = du0 + (T)b * c.ui;
            const T dv = dv0 + (T)b * c.vi;
            const T tu = T(1) - fabs(du);
            const T tv = c.step - c.step * fabs(dv);
            const bool hit = vx.valid && (unsigned)o < (unsigned)n_o && (unsigned)(i0 + b) < (unsigned)n_i &&
                             tu > T(0) && tv > T(0);
            const T w = hit ? tu * tv : T(0);
            const int row = r + b * si;
#pragma unroll
            for (int src = 0; src < V; ++src) {
                const T ws = (LG == 1 || V == 1) ? w : __shfl_sync(0xffffffffu, w, src, LG);
                const int rs = (LG == 1 || V == 1) ? row : __shfl_sync(0xffffffffu, row, src, LG);
                if (ws != T(0)) fma_row_s<T, S, CPL>(acc[src], ws, Gq + (long long)rs * KP);
            }
        }
    }
}

// Four resident blocks (64 registers) pay off while a lane's accumulators are
// 16 floats; larger K keeps three.
template <typename T, typename S, int KP, int LG, int V>
__global__ void __launch_bounds__(kThreads, (KP <= 16 ? 4 : 3))
k_adjoint(const __grid_constant__ AdjParams<T> P, int ns, const S *__restrict__ G, int nj, int nk, int nx,
          int ny, int nz, int ty, int tz, T *__restrict__ gpad, int accumulate, T *__restrict__ gout, int K,
          const double *__restrict__ loss_partials, long long n_partials, double *__restrict__ loss_out,
          LossSlot *loss_slot, unsigned long long loss_seq)
{
    // CTA 0 first sums the forward's loss partials (written by the previous
    // launch on this stream, so visible here without fences) and, given a
    // host-mapped slot, publishes the value there: value, system-scope
    // fence, then the sequence number the host waits for.
    if (loss_out && blockIdx.x == 0) {
        __shared__ double lred[32];
        const double v = sum_fixed_order(loss_partials, n_partials, lred);
        if (threadIdx.x == 0) {
            loss_out[0] = v;
            if (loss_slot) {
                *(volatile double *)&loss_slot->value = v;
                __threadfence_system();
                *(volatile unsigned long long *)&loss_slot->seq = loss_seq;
            }
        }
    }
    constexpr int CPL = KP / LG;
    // A warp's 32/LG lane groups take GZ consecutive z (times GX columns in
    // x); a group owns V voxels adjacent in x, so that the rows the warp
    // reads for one broadcast source are rays of neighbouring voxels and a
    // CTA covers a compact block (8 x 4 x 8 voxels for K = 15: z tiles of 8
    // waste little on volumes whose size is no multiple of 32).  Lane q
    // computes the candidate geometry of voxel q % V (V <= LG; with V < LG
    // lanes repeat a voxel's geometry so that the accumulators, V * CPL per
    // lane, stay in registers for large K).
    constexpr int GPW = 32 / LG;                   // lane groups per warp
    constexpr int GZ = adjoint_gz(LG), GX = GPW / GZ, BY = 4, BX = (kThreads / 32) / BY;

    const int b = blockIdx.x;
    const int bz = b % tz, by = (b / tz) % ty, bx = b / (tz * ty);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = lane / LG, q = lane % LG;
    const int xw = (bx * BX + warp / BY) * (GX * V);   // first x of the warp
    const int x0 = xw + (gw / GZ) * V;             // voxel of source v is (x0 + v, y, z)
    const int y = by * BY + warp % BY;
    const int z = bz * GZ + gw % GZ;
    const int x = x0 + q % V;
    const bool valid = (x < nx) && (y < ny) && (z < nz);
    const T fx = (T)x, fy = (T)y, fz = (T)z;

    T acc[V][CPL];
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
        for (int i = 0; i < CPL; ++i) acc[v][i] = T(0);
    const size_t gstride = (size_t)nj * nk * KP;
    constexpr bool kSmem = std::is_same<T, float>::value && V >= 2;
    __shared__ __align__(16) float s_w[kSmem ? (kThreads / LG) * 36 : 1];
    __shared__ __align__(16) int s_r[kSmem ? (kThreads / LG) * 12 : 1];
    float *wb = s_w + (kSmem ? (threadIdx.x / LG) * 36 : 0);
    int *rb = s_r + (kSmem ? (threadIdx.x / LG) * 12 : 0);

    // Warps whose voxels all lie outside the volume skip the loop as a whole.
    const bool group_live = (xw < nx) && (y < ny) && (bz * GZ < nz);
    if (group_live) {
        for (int si = 0; si < ns; ++si) {
            const AdjProj<T> &c = P.p[si];
            AdjVoxel<T> vx;
            vx.oc = c.oc[0] + c.oc[1] * fx + c.oc[2] * fy + c.oc[3] * fz;
            vx.ic = c.ic[0] + c.ic[1] * fx + c.ic[2] * fy + c.ic[3] * fz;
            vx.bu = c.bu[0] + c.bu[1] * fx + c.bu[2] * fy + c.bu[3] * fz;
            vx.bv = c.bv[0] + c.bv[1] * fx + c.bv[2] * fy + c.bv[3] * fz;
            vx.o0 = (int)(floor(vx.oc - c.ho) + T(1));
            vx.valid = valid;
            const bool outer_j = (c.order >> 16) & 1;
            const int n_o = outer_j ? nj : nk, n_i = outer_j ? nk : nj;
            const int so = outer_j ? nk : 1, sir = outer_j ? 1 : nk;
            const S *Gq = G + (size_t)si * gstride + q * CPL;
#define TT_ADJ_CASE(NO_, NI_)                                                                              \
    case 16 * NO_ + NI_:                                                                                   \
        if constexpr (kSmem) adj_window_sm<S, CPL, KP, LG, V, NO_, NI_>(acc, Gq, vx, c, n_o, n_i, so, sir, wb, rb, q); \
        else adj_window<T, S, CPL, KP, LG, V, NO_, NI_>(acc, Gq, vx, c, n_o, n_i, so, sir);                  \
        break;
            switch (c.shape) {
            TT_ADJ_CASE(1, 1) TT_ADJ_CASE(1, 2) TT_ADJ_CASE(1, 3)
            TT_ADJ_CASE(2, 1) TT_ADJ_CASE(2, 2) TT_ADJ_CASE(2, 3)
            TT_ADJ_CASE(3, 1) TT_ADJ_CASE(3, 2) TT_ADJ_CASE(3, 3)
            default:
                adj_window_any<T, S, CPL, KP, LG, V>(acc, Gq, vx, c, n_o, n_i, so, sir, c.order & 0xff,
                                                     (c.order >> 8) & 0xff);
                break;
            }
#undef TT_ADJ_CASE
        }
    }
    // lane q writes channel chunk q of the group's V voxels
#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int xv = x0 + v;
        if (!(xv < nx && y < ny && z < nz)) continue;
        const long long vox = ((long long)xv * ny + y) * nz + z;
        if (accumulate) {
            const T *prev = gpad + vox * KP + q * CPL;
#pragma unroll
            for (int i = 0; i < CPL; ++i) acc[v][i] += prev[i];
        }
        if (gout) {
            T *o = gout + vox * K;
#pragma unroll
            for (int i = 0; i < CPL; ++i)
                if (q * CPL + i < K) o[q * CPL + i] = acc[v][i];
        } else {
            store_row<T, CPL>(gpad + vox * KP + q * CPL, acc[v], T(1));
        }
    }
}

// ------------------------------------------------------------ launchers

template <typename T, typename S, int L>
cudaError_t launch_forward_L(tt_handle *h, T *Iout, const T *I, const T *W, bool grad, int s0, int s1)
{
    if (s1 < 0) s1 = h->S;
    const int ns = s1 - s0;
    constexpr int K = num_coeffs(L), KP = padded_k(K), LG = lane_group(K);
    // slab order once the padded volume would take more than half of L2
    const long long vol_bytes = (long long)(h->N[0] + 4) * (h->N[1] + 4) * (h->N[2] + 4) * KP * sizeof(S);
    const int slab = vol_bytes > (64LL << 20) ? 1 : 0;
    const T *Bp = (const T *)h->Bp;
    // h->zero_volume: the volume is zero (no packed copy); the kernel gets no
    // volume and marches nothing
    const S *cpad = h->zero_volume ? nullptr : (const S *)h->cpad + h->cpad_origin * KP;
    const S *cpadx = (h->xcopy && !h->zero_volume) ? (const S *)h->cpad + (h->pad_vox + h->cpadx_origin) * KP : nullptr;
    cudaEvent_t ev;
    if constexpr (std::is_same<T, float>::value && std::is_same<S, float>::value && KP == 16) {
        if (h->fwd_staged && !h->zero_volume) {
            const int tiles_k = (h->nk + kStTK - 1) / kStTK, tiles_j = (h->nj + kStTJ - 1) / kStTJ;
            const dim3 grid = slab ? dim3(tiles_k * ns, tiles_j) : dim3(tiles_k * tiles_j, ns);
            const size_t smem = staged_forward_smem(h);
            prof_begin(h, TT_KSLOT_FORWARD, &ev);
            if (grad) {
                auto kern = k_forward_staged<true>;
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kern<<<grid, kStThreads, smem, h->stream>>>(h->geo, h->tmaps, Bp, h->nj, h->nk, h->C, h->CP, tiles_k,
                                                            slab, s0, h->stage_cap, nullptr, I, W, (T *)h->G,
                                                            h->partials);
            } else {
                auto kern = k_forward_staged<false>;
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
                kern<<<grid, kStThreads, smem, h->stream>>>(h->geo, h->tmaps, Bp, h->nj, h->nk, h->C, h->CP, tiles_k,
                                                            slab, s0, h->stage_cap, Iout, nullptr, nullptr, nullptr,
                                                            nullptr);
            }
            cudaError_t e = cudaGetLastError();
            prof_end(h, TT_KSLOT_FORWARD, ev);
            return e;
        }
    }
    constexpr int TK = fwd_tk(LG), TJ = fwd_tj(LG);
    const int tiles_k = (h->nk + TK - 1) / TK, tiles_j = (h->nj + TJ - 1) / TJ;
    const dim3 grid = slab ? dim3(tiles_k * ns, tiles_j) : dim3(tiles_k * tiles_j, ns);
    const size_t smem = (size_t)h->CP * KP * sizeof(T);
    prof_begin(h, TT_KSLOT_FORWARD, &ev);
    if (grad) {
        auto kern = k_forward<T, S, KP, LG, true>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, kFwdThreads, smem, h->stream>>>(h->geo, cpad, cpadx, Bp, h->nj, h->nk, h->C, h->CP, tiles_k, slab, s0,
                                                 nullptr, I, W, (T *)h->G, h->partials);
    } else {
        auto kern = k_forward<T, S, KP, LG, false>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<grid, kFwdThreads, smem, h->stream>>>(h->geo, cpad, cpadx, Bp, h->nj, h->nk, h->C, h->CP, tiles_k, slab, s0,
                                                 Iout, nullptr, nullptr, nullptr, nullptr);
    }
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_FORWARD, ev);
    return e;
}

template <typename T, typename S, int L>
cudaError_t launch_backcontract_L(tt_handle *h, const T *R)
{
    constexpr int K = num_coeffs(L), KP = padded_k(K), LG = lane_group(K);
    constexpr int RAYS = kThreads / LG;
    const long long npix = h->npix();
    const unsigned blocks = (unsigned)((npix + RAYS - 1) / RAYS);
    cudaEvent_t ev;
    prof_begin(h, TT_KSLOT_BACKCONTRACT, &ev);
    k_backcontract<T, S, KP, LG><<<blocks, kThreads, 0, h->stream>>>((const T *)h->Bp, R, (T *)h->G, npix,
                                                                    h->nj * h->nk, h->C, h->CP);
    cudaError_t e = cudaGetLastError();
    prof_end(h, TT_KSLOT_BACKCONTRACT, ev);
    return e;
}

template <typename T, typename S, int L>
cudaError_t launch_adjoint_L(tt_handle *h, T *g, bool reduce_loss)
{
    // For K <= 8 a single lane owns a voxel and reads its whole (32-byte) G
    // row: no candidate exchange, measured 7% faster than two-lane groups.
    // (one lane per voxel for K = 15 as well was measured 0.37 -> 0.50 ms
    // at 64^3: the lane's 16 channels cost the shared weight exchange's
    // savings back in wavefronts)
    constexpr int K = num_coeffs(L), KP = padded_k(K), LG = K <= 8 ? 1 : lane_group(K), V = adjoint_voxels(KP, LG);
    constexpr int GZ = adjoint_gz(LG), BXT = (kThreads / 32 / 4) * (32 / LG / GZ) * V, BY = 4;
    const int tx = (h->N[0] + BXT - 1) / BXT, ty = (h->N[1] + BY - 1) / BY, tz = (h->N[2] + GZ - 1) / GZ;
    const std::vector<AdjParams<T>> &chunks = adj_params<T>(h);
    const T *G = (const T *)h->G;           // G is kept in T for every storage type
    cudaError_t e = cudaSuccess;
    const int nchunk = (int)chunks.size();
    for (int ci = 0; ci < nchunk && e == cudaSuccess; ++ci) {
        const int s0 = ci * AdjParams<T>::kMax;
        const int ns = std::min(AdjParams<T>::kMax, h->S - s0);
        const bool last = ci == nchunk - 1;
        cudaEvent_t ev;
        prof_begin(h, TT_KSLOT_ADJOINT, &ev);
        k_adjoint<T, T, KP, LG, V><<<(unsigned)(tx * ty * tz), kThreads, 0, h->stream>>>(
            chunks[ci], ns, G + (size_t)s0 * h->nj * h->nk * KP, h->nj, h->nk, h->N[0], h->N[1], h->N[2], ty, tz,
            (T *)h->gpad, ci > 0 ? 1 : 0, last ? g : nullptr, h->K, h->partials, h->n_fwd_ctas,
            (reduce_loss && ci == 0) ? h->loss_dev : nullptr,
            (reduce_loss && ci == 0 && h->loss_publish) ? h->loss_slot_dev : nullptr, h->loss_publish);
        e = cudaGetLastError();
        prof_end(h, TT_KSLOT_ADJOINT, ev);
    }
    return e;
}

// Instantiates the three launchers of one (T, S) pair for every band limit.
#define TT_INSTANTIATE_PROJECTORS(T, S)                                                        \
    template <>                                                                                \
    cudaError_t launch_forward<T, S>(tt_handle * h, T * Iout, const T *I, const T *W, bool grad, \
                                     int s0, int s1)                                            \
    {                                                                                          \
        switch (h->L) {                                                                        \
        case 0: return launch_forward_L<T, S, 0>(h, Iout, I, W, grad, s0, s1);                 \
        case 2: return launch_forward_L<T, S, 2>(h, Iout, I, W, grad, s0, s1);                 \
        case 4: return launch_forward_L<T, S, 4>(h, Iout, I, W, grad, s0, s1);                 \
        case 6: return launch_forward_L<T, S, 6>(h, Iout, I, W, grad, s0, s1);                 \
        case 8: return launch_forward_L<T, S, 8>(h, Iout, I, W, grad, s0, s1);                 \
        case 10: return launch_forward_L<T, S, 10>(h, Iout, I, W, grad, s0, s1);               \
        case 12: return launch_forward_L<T, S, 12>(h, Iout, I, W, grad, s0, s1);               \
        default: return cudaErrorInvalidValue;                                                 \
        }                                                                                      \
    }                                                                                          \
    template <>                                                                                \
    cudaError_t launch_backcontract<T, S>(tt_handle * h, const T *R)                           \
    {                                                                                          \
        switch (h->L) {                                                                        \
        case 0: return launch_backcontract_L<T, S, 0>(h, R);                                   \
        case 2: return launch_backcontract_L<T, S, 2>(h, R);                                   \
        case 4: return launch_backcontract_L<T, S, 4>(h, R);                                   \
        case 6: return launch_backcontract_L<T, S, 6>(h, R);                                   \
        case 8: return launch_backcontract_L<T, S, 8>(h, R);                                   \
        case 10: return launch_backcontract_L<T, S, 10>(h, R);                                 \
        case 12: return launch_backcontract_L<T, S, 12>(h, R);                                 \
        default: return cudaErrorInvalidValue;                                                 \
        }                                                                                      \
    }                                                                                          \
    template <>                                                                                \
    cudaError_t launch_adjoint<T, S>(tt_handle * h, T * g, bool rl)                            \
    {                                                                                          \
        switch (h->L) {                                                                        \
        case 0: return launch_adjoint_L<T, S, 0>(h, g, rl);                                    \
        case 2: return launch_adjoint_L<T, S, 2>(h, g, rl);                                    \
        case 4: return launch_adjoint_L<T, S, 4>(h, g, rl);                                    \
        case 6: return launch_adjoint_L<T, S, 6>(h, g, rl);                                    \
        case 8: return launch_adjoint_L<T, S, 8>(h, g, rl);                                    \
        case 10: return launch_adjoint_L<T, S, 10>(h, g, rl);                                  \
        case 12: return launch_adjoint_L<T, S, 12>(h, g, rl);                                  \
        default: return cudaErrorInvalidValue;                                                 \
        }                                                                                      \
    }

}  // namespace tt
