// tt_internal.cuh -- shared declarations of libtt (handle, per-projection
// ray constants, kernel launchers).  Host code is C++17, device code sm_103a.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
#include <string>
#include <vector>

#include "../../include/tt.h"

namespace tt {

// Largest band limit with compiled kernels and its coefficient count.
constexpr int kMaxEll = 12;
constexpr int kMaxSeg = 64;
constexpr int kQuadNodes = 32;      // Gauss-Legendre nodes per detector segment
constexpr int kThreads = 256;       // threads per CTA of the adjoint and the other projector kernels
// Threads of a forward CTA and the ray tile it marches: fwd_tk(LG) rays along
// k (fastest) times fwd_tj(LG) along j, lane_group(K) lanes per ray (8 x 8
// rays at K = 15; 512- and 1024-thread tiles of 16 x 8 and 16 x 16 rays were
// measured 5% and 20% slower at 64^3).
constexpr int kFwdThreads = 256;
__host__ __device__ constexpr int fwd_rays(int LG) { return kFwdThreads / LG; }
__host__ __device__ constexpr int fwd_tk(int LG) { return fwd_rays(LG) >= 256 ? 16 : 8; }
__host__ __device__ constexpr int fwd_tj(int LG) { return fwd_rays(LG) / fwd_tk(LG); }

// Staged forward march (FP32 storage, 16 padded channels): a CTA of eight
// consumer warps and one copy warp marches a tile of kStTJ x kStTK rays with
// its taps read from a ring of shared-memory stages, one plane's box of
// padded-volume voxels per stage, moved by one tensor copy.  The ring holds
// kStRing boxes of the largest size over the projections; a projection with
// smaller boxes runs as many stages as fit, up to kStMaxDepth.  kStEps
// (voxels) widens the box against the rounding of the ray coordinates.
constexpr int kStTJ = 8, kStTK = 16, kStRing = 3, kStMaxDepth = 8;
constexpr int kStConsumers = 256, kStThreads = kStConsumers + 32;
constexpr float kStEps = 1.0f / 64;
constexpr long long kStMaxSmem = 200 * 1024;   // dynamic shared memory the ring may take (one CTA per SM)
constexpr int kStMaxRv = 32;                   // box width along v: 8 x 16 B words per voxel, at most 256 words

// An opaque tensor-map object (the driver's 128-byte, 64-byte aligned
// descriptor of a tiled tensor copy), kept in device memory per projection.
struct alignas(64) TmaDesc {
    unsigned char bytes[128];
};
// Forward kernels a handle can run (tt_set_forward_kernel).
enum { kFwdAuto = 0, kFwdL1 = 1, kFwdStaged = 2 };

// Lane-group width (lanes that share one ray or one voxel, each holding
// KP/LG channels) and padded channel count for a band limit.
__host__ __device__ constexpr int lane_group(int K) { return K <= 4 ? 1 : (K <= 8 ? 2 : 4); }
__host__ __device__ constexpr int padded_k(int K) {
    return ((K + 4 * lane_group(K) - 1) / (4 * lane_group(K))) * (4 * lane_group(K));
}
__host__ __device__ constexpr int num_coeffs(int L) { return (L + 1) * (L + 2) / 2; }
// Voxels a lane group of the adjoint owns: all LG while a lane's accumulators
// (V * KP / LG) fit in 16 registers' worth of channels, else as many as keep
// them within 24 (one for the largest K).
// Lane groups of an adjoint warp along z, the rest side by side in x: eight
// (a warp covers 8 z x 32 / (8 LG) x-columns of V voxels each), all 32 for
// one-lane groups (measured 3% faster for those than 8 z x 4 x).
__host__ __device__ constexpr int adjoint_gz(int LG) { return LG == 1 ? 32 : (32 / LG < 8 ? 32 / LG : 8); }
__host__ __device__ constexpr int adjoint_voxels(int KP, int LG)
{
    return KP / LG <= 4 ? LG : ((24 / (KP / LG)) < 1 ? 1 : ((24 / (KP / LG)) > LG ? LG : 24 / (KP / LG)));
}

// Per-projection constants of the Joseph discretisation, in voxel-index
// units (computed on the host in FP64 from Eq. real_space_geom).
//   plane p (index along the main axis m), ray (j,k):
//     u(j,k,p) = u0 + j*uj + k*uk + p*up   (continuous index along axis u)
//     v(j,k,p) = v0 + j*vj + k*vk + p*vp   (continuous index along axis v)
//   adjoint: the detector point whose ray crosses plane p at voxel (U,V) is
//     jc = jc0 + jU*U + jV*V + jP*p,  kc = kc0 + kU*U + kV*V + kP*p,
//   and every ray that has (U,V) as a bilinear tap lies in
//     |j - jc| < hj, |k - kc| < hk   (the bounding box of the parallelogram
//   |du| < 1, |dv| < 1 in detector coordinates).
struct ProjGeom {
    double u0, uj, uk, up;
    double v0, vj, vk, vp;
    double step;              // a / |p_s,m|
    double jc0, jU, jV, jP;
    double kc0, kU, kV, kP;
    double hj, hk;            // half extents in j and k of the rays around a voxel (|du|, |dv| < 1)
    int m, u, v;              // main and transverse axes (0=x, 1=y, 2=z)
    int Nm, Nu, Nv;
    int sm, su, sv;           // strides of the axes in the padded volume copy the projection reads
    int copy;                 // 0: cpad (z innermost), 1: the x-innermost copy; sv == 1 in both
    // Staged forward: the box of one plane is st_ru rows (along u) of st_rv
    // voxels (along v); st_umid: u is the middle axis (y) of the volume copy,
    // else its outer axis.
    int st_ru, st_rv, st_umid;
};

// Per-projection constants of the adjoint gather in the element type.  The
// candidate rays of a voxel are enumerated over an outer detector axis o and
// an inner axis i ((o, i) = (k, j), or (j, k) when bit 16 of order is set):
//   oc = oc[0] + oc[1] x + oc[2] y + oc[3] z   continuous outer coordinate of
//                                              the voxel centre (likewise ic)
//   du(o,i) = bu(x,y,z) + o uo + i ui,  dv(o,i) = bv(x,y,z) + o vo + i vi
//   columns o = o0 ... o0 + NO - 1,  o0 = floor(oc - ho) + 1
//   column o: i = i0 ... i0 + NI - 1,
//             i0 = floor(ic + max(au + lu (o - oc), av + lv (o - oc))) + 1
// shape = 16 * NO + NI when both are <= 3 (unrolled loops), else 0;
// order = NO | NI << 8 | outer_is_j << 16.
template <typename T>
struct AdjProj {
    T oc[4], ic[4], bu[4], bv[4];
    T uo, ui, vo, vi, ho, au, lu, av, lv, step;
    int shape, order;
};

// Kernel-parameter block holding the constants of up to kMax projections
// (kept under the 32 KB kernel-parameter limit).
template <typename T>
struct AdjParams {
    static constexpr int kMax = sizeof(T) == 4 ? 256 : 128;
    AdjProj<T> p[kMax];
};

struct LossSlot {
    double value;
    unsigned long long seq;
};

struct Profile {
    struct Pending {
        cudaEvent_t begin, end;
        int slot;
        bool free_end;                 // false when `end` is also the next pair's begin
    };
    bool enabled = false;
    // Inside a chain of back-to-back launches on the stream (nothing else
    // enqueued between them), a launch's end event is the next one's begin.
    bool chain = false;
    cudaEvent_t last_end = nullptr;
    std::deque<Pending> pending;       // recorded pairs, oldest first, not yet folded into the totals
    std::vector<cudaEvent_t> free_events;
    double total_ms[TT_KSLOT_COUNT] = {};
    long long launches[TT_KSLOT_COUNT] = {};
};

}  // namespace tt

struct tt_handle {
    tt_precision prec;
    int dev;
    int n_sm = 0;                        // streaming multiprocessors of dev (grid sizing)
    cudaStream_t stream;
    // Recorded on the old stream when tt_set_stream switches streams; the
    // new stream waits on it, so work still in flight on the old stream
    // (an adjoint behind an early-returned loss) finishes with the handle's
    // buffers before the new stream reuses them.
    cudaEvent_t stream_switch = nullptr;
    int N[3];
    int nj, nk, S, L, K, KP, LG, C, CP;
    double a, b, two_theta;
    std::vector<double> inner, outer, joff, koff, seg0, seg1;
    tt_frame frame;
    std::vector<tt::ProjGeom> geo_host;
    tt::ProjGeom *geo = nullptr;        // device [S]
    double *B64 = nullptr;               // device [S][C][K] FP64
    void *Bp = nullptr;                  // device [S][CP][KP], element type, zero padded
    // Padded coefficient volume, two-voxel zero border, channel innermost:
    // [nx+4][ny+4][nz+4][KP] (z innermost) and, when some projection's main
    // axis is z, a second copy [nz+4][ny+4][nx+4][KP] (x innermost) right
    // after it, so that every projection has a transverse axis of stride one
    // and a bilinear tap pair along it is one contiguous 2*KP-element piece.
    void *cpad = nullptr;
    long long cpad_origin = 0;           // voxel offset of (0,0,0) in cpad
    bool zero_volume = false;            // set around a forward launch whose volume is zero (not packed)
    bool xcopy = false;                  // the x-innermost copy exists
    long long pad_vox = 0;               // voxels of one padded copy
    long long cpadx_origin = 0;          // voxel offset of (0,0,0) in the x-innermost copy (from its start)
    void *gpad = nullptr;                // device [nvox][KP]
    void *G = nullptr;                   // device [S][nj][nk][KP]
    double *partials = nullptr;          // device, per-CTA loss partials
    long long n_partials = 0;            // allocated entries
    long long n_fwd_ctas = 0;            // entries the forward kernel writes
    // Staged forward march: voxels of the largest plane box over the
    // projections, rounded up to even (0 when the kernel does not apply),
    // and whether the forward runs it.
    int stage_cap = 0;
    bool fwd_staged = false;
    tt::TmaDesc *tmaps = nullptr;        // device [S]: tensor map of each projection's plane box
    std::vector<tt::TmaDesc> tmaps_host;
    double *red = nullptr;               // device, dot_blocks(h) partials of the regulariser reductions
    double *loss_dev = nullptr;          // device scalars: [0] loss, [1] regulariser value
    double *loss_pinned = nullptr;       // pinned host scalar
    // Page-locked, device-mapped slot where the adjoint's first CTA publishes
    // the loss of a gradient evaluation (value, then sequence number), so
    // that tt_gradient_residual can return it while the adjoint still runs.
    tt::LossSlot *loss_slot_host = nullptr, *loss_slot_dev = nullptr;
    unsigned long long loss_seq = 0;     // last sequence number handed out
    unsigned long long loss_publish = 0; // sequence number the next evaluation publishes (0: none)
    // host-buffer entry point staging (allocated on first use)
    void *hc = nullptr, *hI = nullptr, *hW = nullptr, *hg = nullptr;
    cudaStream_t copy_stream = nullptr;  // host-buffer path: data chunks copied while the forward runs
    cudaStream_t side[2] = {nullptr, nullptr};  // host-buffer path: forward chunks, two at a time
    std::vector<cudaEvent_t> chunk_ready;
    long long launch_count = 0;
    tt::Profile prof;
    std::vector<tt::AdjParams<float>> adj_f32;     // adjoint constants, one block per launch
    std::vector<tt::AdjParams<double>> adj_f64;

    long long nvox() const { return (long long)N[0] * N[1] * N[2]; }
    long long npix() const { return (long long)S * nj * nk; }
    long long ndata() const { return npix() * C; }
    size_t esize() const { return prec == TT_F64 ? 8 : 4; }                 // API element
    size_t ssize() const { return prec == TT_BF16 || prec == TT_F16 ? 2 : esize(); }  // cpad storage
};

namespace tt {

// Compensated FP32 dot-product accumulation (Ogita, Rump & Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005, algorithm Dot2): the
// rounding error of each product comes from an FMA, that of each sum from
// TwoSum, and both are gathered in a second FP32 word.  The result is about
// as accurate as the dot product summed in twice the working precision, at
// FP32 speed (this GPU's FP64 rate is a small fraction of its FP32 rate).
// The _rn intrinsics keep the compiler from contracting the steps.
struct Dot2 {
    float s, c;
};

__device__ __forceinline__ void dot2_add(Dot2 &a, float x, float y)
{
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);          // x y - p, exactly
    const float t = __fadd_rn(a.s, p);
    const float z = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(p, z));   // a.s + p - t, exactly
    a.s = t;
    a.c = __fadd_rn(a.c, __fadd_rn(e, pe));
}

__device__ __forceinline__ double dot2_value(const Dot2 &a) { return (double)a.s + (double)a.c; }

// a += x, compensated (Dot2's summation step alone).
__device__ __forceinline__ void dot2_add1(Dot2 &a, float x)
{
    const float t = __fadd_rn(a.s, x);
    const float z = __fsub_rn(t, a.s);
    const float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, z)), __fsub_rn(x, z));
    a.s = t;
    a.c = __fadd_rn(a.c, e);
}

// (s, c) + (s', c') with the same compensation: TwoSum of the leading parts,
// the error added to the sum of the trailing parts.
__device__ __forceinline__ Dot2 dot2_merge(Dot2 a, Dot2 b)
{
    Dot2 r = a;
    dot2_add1(r, b.s);
    r.c = __fadd_rn(r.c, b.c);
    return r;
}

// Deterministic (fixed-order) block sum of one compensated pair per thread,
// in FP32 arithmetic: a warp tree of dot2_merge, the warps' results merged
// by warp 0.  The one conversion to FP64 happens at the end; on this GPU an
// FP64 shuffle tree per CTA costs tens of times more issue time in the FP64
// pipe than the same tree in FP32.  red: one Dot2 of shared memory per warp;
// the leading barrier lets a CTA call it several times in a row.  Result
// valid on thread 0.
__device__ __forceinline__ double dot2_block_sum(Dot2 v, Dot2 *red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Dot2 o = {__shfl_down_sync(0xffffffffu, v.s, off), __shfl_down_sync(0xffffffffu, v.c, off)};
        v = dot2_merge(v, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    if (w != 0) return 0.0;
    Dot2 t = l < (int)(blockDim.x >> 5) ? red[l] : Dot2{0.f, 0.f};
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const Dot2 o = {__shfl_down_sync(0xffffffffu, t.s, off), __shfl_down_sync(0xffffffffu, t.c, off)};
        t = dot2_merge(t, o);
    }
    return l == 0 ? dot2_value(t) : 0.0;
}

void set_error(const std::string &msg);
tt_status cuda_fail(cudaError_t e, const char *what);
// Problem validation and Gauss-Legendre rule shared by the entry points.
tt_status validate(const tt_problem *P);
void gauss_legendre(int n, double *x, double *w);
// The rows k_basis reads for one projection: R_s^T p, R_s^T q0, R_s^T q90
// (R_s = R_beta(outer angle) R_alpha(inner angle), FP64), 9 doubles.
void basis_frame(const tt_frame &fr, double inner_angle, double outer_angle, double out[9]);

template <typename T>
const std::vector<AdjParams<T>> &adj_params(const tt_handle *h);
template <>
const std::vector<AdjParams<float>> &adj_params<float>(const tt_handle *h);
template <>
const std::vector<AdjParams<double>> &adj_params<double>(const tt_handle *h);

// Bracket a kernel launch with the handle's profiling events.
void prof_begin(tt_handle *h, int slot, cudaEvent_t *ev);
void prof_end(tt_handle *h, int slot, cudaEvent_t ev);
// While alive, the handle's launches share boundary events (the launches it
// covers must be enqueued back to back on the handle's stream).
struct ProfChain {
    tt_handle *h;
    explicit ProfChain(tt_handle *h_);
    ~ProfChain();
    ProfChain(const ProfChain &) = delete;
    ProfChain &operator=(const ProfChain &) = delete;
};

// Kernel launchers (return the launch error, if any).
// Packs c [nvox][K] into the interior of cpad (channels padded to KP).
template <typename T, typename S>
cudaError_t launch_pack(tt_handle *h, const T *c);
template <typename T>
cudaError_t launch_unpack(tt_handle *h, const T *gpad, T *g);
// Projector launchers: arithmetic in T, the coefficient volume cpad stored as
// S (S = T, or a 2-byte type for T = float); the back-contracted residual G
// is T.
// Projections [s0, s1) only (s1 < 0: to the last); the gradient mode writes
// the loss partials of those projections' CTAs.
template <typename T, typename S>
cudaError_t launch_forward(tt_handle *h, T *Iout, const T *I, const T *W, bool grad, int s0 = 0, int s1 = -1);
template <typename T, typename S>
cudaError_t launch_backcontract(tt_handle *h, const T *R);
// g [nvox][K] (unpadded) = exact-transpose gather of G; S above one
// parameter block runs several launches accumulating in h->gpad.
// With reduce_loss the first launch also sums the forward's per-CTA loss
// partials (h->partials, h->n_fwd_ctas) into h->loss_dev[0], in the order of
// launch_reduce, so that the gradient evaluation needs no separate
// reduction launch.
template <typename T, typename S>
cudaError_t launch_adjoint(tt_handle *h, T *g, bool reduce_loss = false);
cudaError_t launch_reduce(tt_handle *h, const double *partials, long long n, double *out,
                          const double *add, double mul);
cudaError_t launch_basis(tt_handle *h, const double *nodes, const double *weights);
template <typename T>
cudaError_t launch_cast_basis(tt_handle *h);

// FP64-accumulated vector kernels for the optimizer.
template <typename T>
cudaError_t vec_dot(tt_handle *h, const T *x, const T *y, long long n, double *partials,
                    double *out, const double *add, double mul);
// y = a*x + b*y with a = ha * (da ? *da : 1), b = hb (y is not read when hb == 0)
template <typename T>
cudaError_t vec_axpby(tt_handle *h, T *y, const T *x, long long n, double ha, const double *da, double hb);
template <typename T>
cudaError_t vec_sub(tt_handle *h, T *out, const T *x, const T *y, long long n);
// Streaming-multiprocessor count of the current device (queried once per
// device ordinal and cached); grids of the grid-stride kernels are capped at
// multiples of it.
int current_sm_count();
// CTAs of the dot-product and regulariser reductions: four per SM.
inline int dot_blocks(const tt_handle *h) { return 4 * h->n_sm; }
// Dynamic shared memory of the staged forward: the stage ring, B_s and 128
// bytes of slack to align the ring.
inline size_t staged_forward_smem(const tt_handle *h)
{
    return (size_t)kStRing * h->stage_cap * 16 * sizeof(float) + (size_t)h->CP * 16 * sizeof(float) + 128;
}

}  // namespace tt
