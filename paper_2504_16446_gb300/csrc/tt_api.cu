// tt_api.cu -- C ABI of libtt: validation, geometry set-up (host, FP64),
// buffer ownership and the orchestration of the kernels on the handle's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "tt_internal.cuh"

namespace tt {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

tt_status cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TT_OUT_OF_MEMORY : TT_CUDA_ERROR;
}

#define TT_CUDA(call, what)                                  \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return ::tt::cuda_fail(_e, what); \
    } while (0)

int current_sm_count()
{
    static std::atomic<int> cache[256];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        (void)cudaGetLastError();
        return 1;
    }
    int n = cache[dev].load(std::memory_order_relaxed);
    if (n < 1) {
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            (void)cudaGetLastError();
            return 1;
        }
        cache[dev].store(n, std::memory_order_relaxed);
    }
    return n;
}

static tt_status invalid(const std::string &msg)
{
    set_error(msg);
    return TT_INVALID_ARG;
}

// Launch timing with CUDA events.  Events come from a free list that is
// filled when profiling is switched on, and before each new launch up to two
// recorded pairs whose end event has completed are folded into the totals,
// so that a long timed loop neither creates events nor grows the list of
// pairs: its cost is two event records and a query or two per launch.
static constexpr size_t kProfileEvents = 256;

// Folds up to max_pairs pairs, oldest first, into the totals.  With wait,
// waits for them; otherwise stops at the first pair still in flight.
static cudaError_t prof_fold(tt_handle *h, bool wait, size_t max_pairs)
{
    auto &P = h->prof;
    for (size_t n = 0; n < max_pairs && !P.pending.empty(); ++n) {
        const tt::Profile::Pending r = P.pending.front();
        if (!wait) {
            const cudaError_t q = cudaEventQuery(r.end);
            if (q == cudaErrorNotReady) {
                (void)cudaGetLastError();   // "not ready" is no error: keep it out of the launch checks
                break;
            }
            if (q != cudaSuccess) return q;
        }
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.end);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.begin, r.end);
        if (e != cudaSuccess) return e;
        P.total_ms[r.slot] += ms;
        P.launches[r.slot] += 1;
        P.free_events.push_back(r.begin);
        if (r.free_end) P.free_events.push_back(r.end);
        P.pending.pop_front();
    }
    return cudaSuccess;
}

static cudaEvent_t prof_event(tt_handle *h)
{
    auto &P = h->prof;
    prof_fold(h, false, 2);
    if (P.free_events.empty()) {
        cudaEvent_t e;
        return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
    }
    cudaEvent_t e = P.free_events.back();
    P.free_events.pop_back();
    return e;
}

void prof_begin(tt_handle *h, int slot, cudaEvent_t *ev)
{
    (void)slot;
    ++h->launch_count;
    *ev = nullptr;
    auto &P = h->prof;
    if (!P.enabled) return;
    if (P.chain && P.last_end) {
        // the previous launch's end event, the back pair of the list
        *ev = P.last_end;
        P.pending.back().free_end = false;
        P.last_end = nullptr;
        return;
    }
    cudaEvent_t e = prof_event(h);
    if (!e) return;
    cudaEventRecord(e, h->stream);
    *ev = e;
}

void prof_end(tt_handle *h, int slot, cudaEvent_t ev)
{
    if (!h->prof.enabled || ev == nullptr) return;
    cudaEvent_t e = prof_event(h);
    if (!e) {
        h->prof.free_events.push_back(ev);
        return;
    }
    cudaEventRecord(e, h->stream);
    h->prof.pending.push_back({ev, e, slot, true});
    h->prof.last_end = h->prof.chain ? e : nullptr;
}

ProfChain::ProfChain(tt_handle *h_) : h(h_)
{
    h->prof.chain = true;
    h->prof.last_end = nullptr;
}

ProfChain::~ProfChain()
{
    h->prof.chain = false;
    h->prof.last_end = nullptr;
}

// ---------------------------------------------------------------- geometry

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return std::sqrt(dot3(a, a)); }

// Right-handed rotation by angle t about the unit axis n (Rodrigues).
static void axis_angle(const double *n, double t, double R[9])
{
    const double c = std::cos(t), s = std::sin(t), C1 = 1.0 - c;
    const double x = n[0], y = n[1], z = n[2];
    R[0] = c + x * x * C1;     R[1] = x * y * C1 - z * s; R[2] = x * z * C1 + y * s;
    R[3] = y * x * C1 + z * s; R[4] = c + y * y * C1;     R[5] = y * z * C1 - x * s;
    R[6] = z * x * C1 - y * s; R[7] = z * y * C1 + x * s; R[8] = c + z * z * C1;
}

static void matmul3(const double A[9], const double B[9], double out[9])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) out[3 * r + c] = A[3 * r] * B[c] + A[3 * r + 1] * B[3 + c] + A[3 * r + 2] * B[6 + c];
}

// out = R^T v
static void apply_transpose(const double R[9], const double *v, double *out)
{
    for (int c = 0; c < 3; ++c) out[c] = R[c] * v[0] + R[3 + c] * v[1] + R[6 + c] * v[2];
}

struct Frames { double p[3], j[3], k[3], q0[3], q90[3]; };

// Sample-frame vectors R_s^T v of one projection, R_s = R_beta(beta) R_alpha(alpha).
static Frames frames_of(const tt_frame &fr, double alpha, double beta)
{
    double ax[3], bx[3];
    const double na = norm3(fr.inner_axis), nb = norm3(fr.outer_axis);
    for (int t = 0; t < 3; ++t) { ax[t] = fr.inner_axis[t] / na; bx[t] = fr.outer_axis[t] / nb; }
    double Ra[9], Rb[9], R[9];
    axis_angle(ax, alpha, Ra);
    axis_angle(bx, beta, Rb);
    matmul3(Rb, Ra, R);                      // R_s = R_beta(beta) R_alpha(alpha)
    Frames f;
    apply_transpose(R, fr.p, f.p);
    apply_transpose(R, fr.j, f.j);
    apply_transpose(R, fr.k, f.k);
    apply_transpose(R, fr.q0, f.q0);
    apply_transpose(R, fr.q90, f.q90);
    return f;
}

static Frames projection_frames(const tt_handle *h, int s) { return frames_of(h->frame, h->inner[s], h->outer[s]); }

void basis_frame(const tt_frame &fr, double alpha, double beta, double out[9])
{
    const Frames f = frames_of(fr, alpha, beta);
    for (int t = 0; t < 3; ++t) { out[t] = f.p[t]; out[3 + t] = f.q0[t]; out[6 + t] = f.q90[t]; }
}

// Main axis of the Joseph march: the largest |p_s| component, ties to the
// smallest axis.
static int main_axis(const double *d)
{
    const double mx = std::fmax(std::fabs(d[0]), std::fmax(std::fabs(d[1]), std::fabs(d[2])));
    int m = 0;
    while (std::fabs(d[m]) < (1.0 - 1e-12) * mx) ++m;
    return m;
}

static ProjGeom make_geom(const tt_handle *h, int s)
{
    const Frames f = projection_frames(h, s);
    const double *d = f.p;
    const int m = main_axis(d);
    // The transverse axis v is the innermost axis of the copy the projection
    // reads: z for m = x, y (cpad), x for m = z (the x-innermost copy).
    const int copy = (m == 2) ? 1 : 0;
    const int u = (m == 0) ? 1 : (m == 1 ? 0 : 1);
    const int v = (m == 2) ? 0 : 2;
    const int stride_z[3] = {(h->N[1] + 4) * (h->N[2] + 4), h->N[2] + 4, 1};
    const int stride_x[3] = {1, h->N[0] + 4, (h->N[1] + 4) * (h->N[0] + 4)};
    const int *stride = copy ? stride_x : stride_z;
    const double ba = h->b / h->a;
    const double cj = 0.5 * (h->nj - 1) + h->joff[s], ck = 0.5 * (h->nk - 1) + h->koff[s];
    const double hm = 0.5 * (h->N[m] - 1), hu = 0.5 * (h->N[u] - 1), hv = 0.5 * (h->N[v] - 1);
    ProjGeom g;
    g.m = m; g.u = u; g.v = v;
    g.copy = copy;
    g.Nm = h->N[m]; g.Nu = h->N[u]; g.Nv = h->N[v];
    g.sm = stride[m]; g.su = stride[u]; g.sv = stride[v];
    g.up = d[u] / d[m];
    g.vp = d[v] / d[m];
    g.uj = ba * (f.j[u] - f.j[m] * g.up);
    g.uk = ba * (f.k[u] - f.k[m] * g.up);
    g.vj = ba * (f.j[v] - f.j[m] * g.vp);
    g.vk = ba * (f.k[v] - f.k[m] * g.vp);
    g.u0 = hu - cj * g.uj - ck * g.uk - hm * g.up;
    g.v0 = hv - cj * g.vj - ck * g.vk - hm * g.vp;
    g.step = h->a / std::fabs(d[m]);
    // inverse of the pixel -> plane map [[uj uk],[vj vk]]
    const double det = g.uj * g.vk - g.uk * g.vj;
    const double i00 = g.vk / det, i01 = -g.uk / det, i10 = -g.vj / det, i11 = g.uj / det;
    g.jU = i00; g.jV = i01; g.jP = -(i00 * g.up + i01 * g.vp); g.jc0 = -(i00 * g.u0 + i01 * g.v0);
    g.kU = i10; g.kV = i11; g.kP = -(i10 * g.up + i11 * g.vp); g.kc0 = -(i10 * g.u0 + i11 * g.v0);
    g.hj = std::fabs(i00) + std::fabs(i01);
    g.hk = std::fabs(i10) + std::fabs(i11);
    return g;
}

// Number of integers an open interval of length L can hold (L within FP
// rounding of an integer n counts as n: a point that only rounding puts
// inside has weight within rounding of zero).
static int points_in(double L) { return std::max(1, (int)std::ceil(L - 1e-9)); }

// Lower edge of the inner coordinate, relative to the voxel centre, as a
// function of the outer offset d: the constraint |ci di + co d| < 1 gives
// di > -1/|ci| - (co/ci) d.  A vanishing ci leaves the inner axis unbounded
// by this constraint.
static void inner_edge(double ci, double co, double &offset, double &slope, double &length)
{
    if (std::fabs(ci) < 1e-12) { offset = -1e30; slope = 0.0; length = 1e30; return; }
    offset = -1.0 / std::fabs(ci);
    slope = -co / ci;
    length = 2.0 / std::fabs(ci);
}

template <typename T>
static AdjProj<T> adj_proj(const ProjGeom &g)
{
    double jc[4] = {g.jc0, 0, 0, 0}, kc[4] = {g.kc0, 0, 0, 0}, bu[4] = {g.u0, 0, 0, 0}, bv[4] = {g.v0, 0, 0, 0};
    jc[1 + g.m] += g.jP; jc[1 + g.u] += g.jU; jc[1 + g.v] += g.jV;
    kc[1 + g.m] += g.kP; kc[1 + g.u] += g.kU; kc[1 + g.v] += g.kV;
    bu[1 + g.m] += g.up; bu[1 + g.u] -= 1.0;
    bv[1 + g.m] += g.vp; bv[1 + g.v] -= 1.0;
    // the two enumeration orders: outer k / inner j, and outer j / inner k
    double au[2], lu[2], av[2], lv[2];
    int no[2], ni[2];
    for (int t = 0; t < 2; ++t) {
        const bool outer_j = t == 1;
        const double ui = outer_j ? g.uk : g.uj, uo = outer_j ? g.uj : g.uk;
        const double vi = outer_j ? g.vk : g.vj, vo = outer_j ? g.vj : g.vk;
        double Lu, Lv;
        inner_edge(ui, uo, au[t], lu[t], Lu);
        inner_edge(vi, vo, av[t], lv[t], Lv);
        const double hi = outer_j ? g.hk : g.hj, ho = outer_j ? g.hj : g.hk;
        no[t] = points_in(2.0 * ho);
        ni[t] = points_in(std::min(std::min(Lu, Lv), 2.0 * hi));
    }
    const int t = (no[1] * ni[1] < no[0] * ni[0]) ? 1 : 0;
    const bool outer_j = t == 1;
    AdjProj<T> a;
    for (int i = 0; i < 4; ++i) {
        a.oc[i] = (T)(outer_j ? jc[i] : kc[i]);
        a.ic[i] = (T)(outer_j ? kc[i] : jc[i]);
        a.bu[i] = (T)bu[i];
        a.bv[i] = (T)bv[i];
    }
    a.uo = (T)(outer_j ? g.uj : g.uk); a.ui = (T)(outer_j ? g.uk : g.uj);
    a.vo = (T)(outer_j ? g.vj : g.vk); a.vi = (T)(outer_j ? g.vk : g.vj);
    a.ho = (T)(outer_j ? g.hj : g.hk);
    a.au = (T)au[t]; a.lu = (T)lu[t]; a.av = (T)av[t]; a.lv = (T)lv[t];
    a.step = (T)g.step;
    a.shape = (no[t] <= 3 && ni[t] <= 3) ? 16 * no[t] + ni[t] : 0;
    a.order = no[t] | (ni[t] << 8) | ((outer_j ? 1 : 0) << 16);
    return a;
}

template <typename T>
static void build_adj_params(const tt_handle *h, std::vector<AdjParams<T>> &out)
{
    const int per = AdjParams<T>::kMax;
    out.assign((h->S + per - 1) / per, AdjParams<T>());
    for (int s = 0; s < h->S; ++s) out[s / per].p[s % per] = adj_proj<T>(h->geo_host[s]);
}

template <>
const std::vector<AdjParams<float>> &adj_params<float>(const tt_handle *h) { return h->adj_f32; }
template <>
const std::vector<AdjParams<double>> &adj_params<double>(const tt_handle *h) { return h->adj_f64; }

// Gauss-Legendre nodes/weights on [-1, 1] (Newton on the three-term recurrence).
void gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double z = std::cos(pi * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int l = 2; l <= n; ++l) {
                const double p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l;
                p0 = p1; p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-15) {
                p0 = 1.0; p1 = z;
                for (int l = 2; l <= n; ++l) {
                    const double p2 = ((2 * l - 1) * z * p1 - (l - 1) * p0) / l;
                    p0 = p1; p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static bool finite_all(const double *a, int n)
{
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

tt_status validate(const tt_problem *P)
{
    if (!P) return invalid("tt_create: null problem");
    if (P->nx < 1 || P->ny < 1 || P->nz < 1) return invalid("volume shape must be >= 1 in every axis");
    if ((long long)P->nx * P->ny * P->nz > (1LL << 31) / 128) return invalid("volume too large");
    if (P->nj < 1 || P->nk < 1) return invalid("nj, nk must be >= 1");
    if (P->n_proj < 1 || P->n_proj > 65535) return invalid("n_proj must be in [1, 65535]");
    if (P->ell_max < 0 || (P->ell_max & 1)) return invalid("ell_max must be even and >= 0");
    if (P->n_seg < 1 || P->n_seg > kMaxSeg) return invalid("n_seg must be in [1, 64]");
    if (!P->inner_angle || !P->outer_angle || !P->seg_start || !P->seg_end)
        return invalid("angle and segment arrays must not be NULL");
    if (!finite_all(P->inner_angle, P->n_proj) || !finite_all(P->outer_angle, P->n_proj))
        return invalid("rotation/tilt angles must be finite");
    if ((P->j_offset && !finite_all(P->j_offset, P->n_proj)) || (P->k_offset && !finite_all(P->k_offset, P->n_proj)))
        return invalid("offsets must be finite");
    for (int c = 0; c < P->n_seg; ++c)
        if (!std::isfinite(P->seg_start[c]) || !std::isfinite(P->seg_end[c]) || !(P->seg_end[c] > P->seg_start[c]))
            return invalid("every segment needs finite seg_end > seg_start");
    if (!(P->voxel_size > 0) || !(P->step_size > 0) || !std::isfinite(P->voxel_size) || !std::isfinite(P->step_size))
        return invalid("voxel_size and step_size must be positive and finite");
    if (P->step_size < 0.02 * P->voxel_size)
        return invalid("step_size (detector pixel) must be at least 1/50 of voxel_size");
    if (!std::isfinite(P->two_theta)) return invalid("two_theta must be finite");
    const tt_frame &f = P->frame;
    const double *unit[5] = {f.p, f.j, f.k, f.q0, f.q90};
    const char *names[5] = {"p", "j", "k", "q0", "q90"};
    for (int t = 0; t < 5; ++t)
        if (!(std::fabs(norm3(unit[t]) - 1.0) < 1e-9)) return invalid(std::string("frame vector ") + names[t] + " is not a unit vector");
    if (!(norm3(f.inner_axis) > 1e-12) || !(norm3(f.outer_axis) > 1e-12) || !std::isfinite(norm3(f.inner_axis)) ||
        !std::isfinite(norm3(f.outer_axis)))
        return invalid("rotation axes must be non-zero and finite");
    if (std::fabs(dot3(f.p, f.j)) > 1e-9 || std::fabs(dot3(f.p, f.k)) > 1e-9 || std::fabs(dot3(f.j, f.k)) > 1e-9)
        return invalid("p, j, k must be mutually orthogonal");
    if (std::fabs(dot3(f.p, f.q0)) > 1e-9 || std::fabs(dot3(f.p, f.q90)) > 1e-9 || std::fabs(dot3(f.q0, f.q90)) > 1e-9)
        return invalid("q0, q90 must be orthogonal to each other and to p");
    return TT_OK;
}

static void free_handle(tt_handle *h)
{
    if (!h) return;
    cudaFree(h->geo); cudaFree(h->tmaps); cudaFree(h->B64); cudaFree(h->Bp); cudaFree(h->cpad); cudaFree(h->gpad);
    cudaFree(h->G); cudaFree(h->partials); cudaFree(h->loss_dev); cudaFree(h->red);
    cudaFree(h->hc); cudaFree(h->hI); cudaFree(h->hW); cudaFree(h->hg);
    for (cudaEvent_t e : h->chunk_ready) cudaEventDestroy(e);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    for (cudaStream_t t : h->side)
        if (t) cudaStreamDestroy(t);
    if (h->stream_switch) cudaEventDestroy(h->stream_switch);
    if (h->loss_pinned) cudaFreeHost(h->loss_pinned);
    if (h->loss_slot_host) cudaFreeHost(h->loss_slot_host);
    for (const auto &r : h->prof.pending) {
        cudaEventDestroy(r.begin);
        if (r.free_end) cudaEventDestroy(r.end);
    }
    for (cudaEvent_t e : h->prof.free_events) cudaEventDestroy(e);
    delete h;
}

static long long forward_ctas(const tt_handle *h, bool staged)
{
    const int TK = staged ? kStTK : fwd_tk(h->LG), TJ = staged ? kStTJ : fwd_tj(h->LG);
    return (long long)((h->nk + TK - 1) / TK) * ((h->nj + TJ - 1) / TJ) * h->S;
}

// Box of the staged forward for projection g: a tile's rays span W = (TJ - 1)
// |uj| + (TK - 1)|uk| in u at every plane (the rays are parallel), and the
// rows floor(c) and floor(c) + 1 for c within kStEps of that span number at
// most floor(W + 2 kStEps) + 3; likewise in v.  1e-3 voxels more covers the
// FP32 rounding of the ray coordinates.
static void stage_box(const ProjGeom &g, int nj, int nk, int &ru, int &rv)
{
    const double tj = std::min(kStTJ, nj) - 1, tk = std::min(kStTK, nk) - 1;
    const double m = 2.0 * kStEps + 1e-3;
    ru = (int)std::floor(tj * std::fabs(g.uj) + tk * std::fabs(g.uk) + m) + 3;
    rv = (int)std::floor(tj * std::fabs(g.vj) + tk * std::fabs(g.vk) + m) + 3;
}

void *driver_tensor_map_encoder()
{
    static void *fn = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        (void)cudaGetLastError();
        return p;
    }();
    return fn;
}

// Tensor map of projection g's plane box over the padded volume copy it
// reads.  The copy is viewed as a 3-D tensor of 8-byte words: the innermost
// dimension merges v and the 16 channels (8 words per voxel), then the middle
// axis (y) and the outer axis (x for the z-innermost copy, z for the other).
// The box is st_rv voxels wide and st_ru rows long along u (the middle or the
// outer axis), one plane thick along the main axis; coordinates outside the
// tensor read as zero.
static bool encode_box_map(const tt_handle *h, const ProjGeom &g, TmaDesc *out)
{
    const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(driver_tensor_map_encoder());
    if (!enc) return false;
    const int nin = g.copy ? h->N[0] : h->N[2], nout = g.copy ? h->N[2] : h->N[0];
    const cuuint64_t dims[3] = {(cuuint64_t)8 * (nin + 4), (cuuint64_t)(h->N[1] + 4), (cuuint64_t)(nout + 4)};
    const cuuint64_t strides[2] = {(cuuint64_t)(nin + 4) * 64, (cuuint64_t)(nin + 4) * (h->N[1] + 4) * 64};
    const cuuint32_t box[3] = {(cuuint32_t)(8 * g.st_rv), (cuuint32_t)(g.st_umid ? g.st_ru : 1),
                               (cuuint32_t)(g.st_umid ? 1 : g.st_ru)};
    const cuuint32_t elem[3] = {1, 1, 1};
    void *base = (char *)h->cpad + (g.copy ? h->pad_vox * 64 : 0);
    static_assert(sizeof(TmaDesc) == sizeof(CUtensorMap), "tensor-map size");
    CUtensorMap m;
    const CUresult r = enc(&m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, base, dims, strides, box, elem,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    std::memcpy(out, &m, sizeof(m));
    return true;
}

// The staged forward applies to FP32 storage with 16 padded channels when
// kStRing boxes of the largest size fit in the shared memory of one CTA, every
// box is at most kStMaxRv voxels wide, and the driver encodes the tensor maps.
// Sets each projection's box, the ring size and the maps (enqueued on the
// handle's stream).
static void plan_forward(tt_handle *h)
{
    h->stage_cap = 0;
    if (h->prec != TT_F32 || h->KP != 16) return;
    long long cap = 0;
    bool fits = true;
    for (ProjGeom &g : h->geo_host) {
        stage_box(g, h->nj, h->nk, g.st_ru, g.st_rv);
        g.st_umid = g.u == 1 ? 1 : 0;
        fits = fits && g.st_rv <= kStMaxRv && g.st_ru <= 256;
        cap = std::max(cap, (long long)((g.st_ru * g.st_rv + 1) & ~1));
    }
    const long long bytes = (long long)kStRing * cap * 16 * 4 + (long long)h->CP * 16 * 4 + 128;
    if (!fits || bytes > kStMaxSmem) return;
    h->tmaps_host.resize(h->S);
    for (int s = 0; s < h->S; ++s)
        if (!encode_box_map(h, h->geo_host[s], &h->tmaps_host[s])) return;
    if (cudaMalloc((void **)&h->tmaps, sizeof(TmaDesc) * h->S) != cudaSuccess ||
        cudaMemcpyAsync(h->tmaps, h->tmaps_host.data(), sizeof(TmaDesc) * h->S, cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    h->stage_cap = (int)cap;
}

// Checks a device pointer argument: non-null, 16-byte aligned.
static bool bad_ptr(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

// Calls f.template operator()<S>() with the storage type S of the handle's
// coefficient volume and G (T itself, or bf16 / f16 for a float handle).
template <typename T, typename F>
static tt_status with_storage(const tt_handle *h, F &&f)
{
    if constexpr (std::is_same<T, double>::value) {
        return f.template operator()<double>();
    } else {
        if (h->prec == TT_BF16) return f.template operator()<__nv_bfloat16>();
        if (h->prec == TT_F16) return f.template operator()<__half>();
        return f.template operator()<float>();
    }
}

template <typename T>
static tt_status project_impl(tt_handle *h, const T *c, T *I)
{
    if (bad_ptr(c) || bad_ptr(I)) return invalid("tt_project: device pointers must be non-null and 16-byte aligned");
    return with_storage<T>(h, [&]<typename S>() -> tt_status {
        const ProfChain chain(h);   // pack, forward and adjoint run back to back
        TT_CUDA((launch_pack<T, S>(h, c)), "pack");
        TT_CUDA((launch_forward<T, S>(h, I, nullptr, nullptr, false)), "forward");
        return TT_OK;
    });
}

template <typename T>
static tt_status adjoint_impl(tt_handle *h, const T *R, T *g)
{
    if (bad_ptr(R) || bad_ptr(g)) return invalid("tt_adjoint: device pointers must be non-null and 16-byte aligned");
    return with_storage<T>(h, [&]<typename S>() -> tt_status {
        TT_CUDA((launch_backcontract<T, S>(h, R)), "backcontract");
        TT_CUDA((launch_adjoint<T, S>(h, g)), "adjoint");
        return TT_OK;
    });
}

}  // namespace tt

using namespace tt;

// While in scope with on = true: the forward launcher projects a zero volume
// (h->zero_volume), which always takes the L1 kernel, so the loss reduction
// reads that kernel's number of partials whichever forward kernel is chosen.
struct ZeroVolume {
    tt_handle *h;
    long long saved;
    ZeroVolume(tt_handle *h_, bool on) : h(h_), saved(h_->n_fwd_ctas)
    {
        if (on) {
            h->zero_volume = true;
            h->n_fwd_ctas = forward_ctas(h, false);
        }
    }
    ~ZeroVolume()
    {
        h->zero_volume = false;
        h->n_fwd_ctas = saved;
    }
};

// Enqueues the gradient-residual evaluation; the loss lands in h->loss_dev.
template <typename T>
tt_status tt_grad_enqueue(tt_handle *h, const T *c, const T *I, const T *W, T *g)
{
    if ((c && bad_ptr(c)) || bad_ptr(I) || (W && bad_ptr(W)) || (g && bad_ptr(g)))
        return invalid("tt_gradient_residual: device pointers must be non-null (c, W, g may be NULL) and 16-byte aligned");
    return with_storage<T>(h, [&]<typename S>() -> tt_status {
        const ProfChain chain(h);   // pack, forward and adjoint run back to back
        // c == NULL: the volume is zero; nothing is packed and the forward
        // kernel skips its march (every projection is exactly zero), so the
        // evaluation is the back-projection of the data alone
        if (c) TT_CUDA((launch_pack<T, S>(h, c)), "pack");
        const ZeroVolume zero(h, c == nullptr);
        TT_CUDA((launch_forward<T, S>(h, nullptr, I, W, true)), "forward");
        // the adjoint's first CTA reduces the loss partials; without a
        // gradient a one-CTA reduction does
        if (g) TT_CUDA((launch_adjoint<T, S>(h, g, true)), "adjoint");
        else TT_CUDA(launch_reduce(h, h->partials, h->n_fwd_ctas, h->loss_dev, nullptr, 1.0), "loss reduce");
        return TT_OK;
    });
}
template tt_status tt_grad_enqueue<float>(tt_handle *, const float *, const float *, const float *, float *);
template tt_status tt_grad_enqueue<double>(tt_handle *, const double *, const double *, const double *, double *);

static tt_status check_finite_loss(double v)
{
    if (!std::isfinite(v)) {
        set_error("loss is not finite (NaN/Inf in the inputs)");
        return TT_NONFINITE;
    }
    return TT_OK;
}

tt_status tt_read_loss(tt_handle *h, double *loss_host);

unsigned long long loss_publish_begin(tt_handle *h)
{
    h->loss_publish = h->loss_slot_host ? ++h->loss_seq : 0;
    return h->loss_publish;
}

// Waits until the loss with sequence number seq is in the mapped slot, or
// until the stream has drained (then the slot must hold it; if it does not,
// the loss is copied as by tt_read_loss).  Errors of the stream are returned.
tt_status read_published_loss(tt_handle *h, unsigned long long seq, double *loss_host)
{
    const volatile LossSlot *slot = h->loss_slot_host;
    for (;;) {
        if (slot->seq == seq) break;
        const cudaError_t q = cudaStreamQuery(h->stream);
        if (q == cudaSuccess) {
            if (slot->seq == seq) break;
            return tt_read_loss(h, loss_host);
        }
        if (q != cudaErrorNotReady) return cuda_fail(q, "stream");
        (void)cudaGetLastError();          // "not ready" is no error
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    const double v = slot->value;
    if (loss_host) *loss_host = v;
    return check_finite_loss(v);
}

tt_status tt_read_loss(tt_handle *h, double *loss_host)
{
    TT_CUDA(cudaMemcpyAsync(h->loss_pinned, h->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, h->stream), "loss copy");
    TT_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    const double v = *h->loss_pinned;
    if (loss_host) *loss_host = v;
    if (!std::isfinite(v)) {
        set_error("loss is not finite (NaN/Inf in the inputs)");
        return TT_NONFINITE;
    }
    return TT_OK;
}

template <typename T>
static tt_status grad_impl(tt_handle *h, const T *c, const T *I, const T *W, T *g, double *loss_host)
{
    if (!loss_host) return invalid("tt_gradient_residual: loss_host must not be NULL");
    // With a gradient, the adjoint's first CTA publishes the loss in the
    // mapped slot and the call returns once it is there; the rest of the
    // adjoint stays in flight on the stream (g is stream-ordered like every
    // device output).
    const unsigned long long seq = g ? loss_publish_begin(h) : 0;
    tt_status st = tt_grad_enqueue<T>(h, c, I, W, g);
    h->loss_publish = 0;
    if (st != TT_OK) return st;
    return seq ? read_published_loss(h, seq, loss_host) : tt_read_loss(h, loss_host);
}

// want = TT_F32 for the float entry points (handles of precision TT_F32,
// TT_BF16 or TT_F16), TT_F64 for the _f64 ones.
static tt_status check_handle(const tt_handle *h, tt_precision want)
{
    if (!h) return invalid("null handle");
    if ((h->prec == TT_F64) != (want == TT_F64))
        return invalid("handle precision does not match the entry point (use the _f64 variants with TT_F64)");
    return TT_OK;
}

extern "C" {

int tt_num_coeffs(int ell_max) { return ell_max < 0 ? 0 : (ell_max + 1) * (ell_max + 2) / 2; }

const char *tt_status_string(tt_status s)
{
    switch (s) {
    case TT_OK: return "TT_OK";
    case TT_INVALID_ARG: return "TT_INVALID_ARG";
    case TT_UNSUPPORTED: return "TT_UNSUPPORTED";
    case TT_OUT_OF_MEMORY: return "TT_OUT_OF_MEMORY";
    case TT_NONFINITE: return "TT_NONFINITE";
    case TT_LINESEARCH_FAILED: return "TT_LINESEARCH_FAILED";
    case TT_CUDA_ERROR: return "TT_CUDA_ERROR";
    }
    return "TT_UNKNOWN";
}

const char *tt_last_error(void) { return g_last_error.c_str(); }

tt_status tt_create(const tt_problem *P, tt_precision prec, void *stream, tt_handle **out)
{
    if (!out) return invalid("tt_create: out must not be NULL");
    *out = nullptr;
    tt_status st = validate(P);
    if (st != TT_OK) return st;
    if (prec != TT_F32 && prec != TT_F64 && prec != TT_BF16 && prec != TT_F16)
        return invalid("precision must be TT_F32, TT_F64, TT_BF16 or TT_F16");
    if (P->ell_max > kMaxEll) {
        set_error("ell_max above 12 has no compiled kernels");
        return TT_UNSUPPORTED;
    }
    tt_handle *h = new (std::nothrow) tt_handle();
    if (!h) return TT_OUT_OF_MEMORY;
    h->prec = prec;
    cudaGetDevice(&h->dev);
    if (cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, h->dev) != cudaSuccess || h->n_sm < 1) {
        delete h;
        set_error("tt_create: cannot query the multiprocessor count of the current device");
        return TT_CUDA_ERROR;
    }
    h->stream = (cudaStream_t)stream;
    if (cudaEventCreateWithFlags(&h->stream_switch, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        set_error("tt_create: cudaEventCreate failed");
        return TT_CUDA_ERROR;
    }
    h->N[0] = P->nx; h->N[1] = P->ny; h->N[2] = P->nz;
    h->nj = P->nj; h->nk = P->nk; h->S = P->n_proj; h->L = P->ell_max; h->C = P->n_seg;
    h->K = num_coeffs(h->L);
    h->KP = padded_k(h->K);
    h->LG = lane_group(h->K);
    h->CP = (h->C + 3) / 4 * 4;
    h->a = P->voxel_size; h->b = P->step_size; h->two_theta = P->two_theta;
    h->frame = P->frame;
    h->inner.assign(P->inner_angle, P->inner_angle + h->S);
    h->outer.assign(P->outer_angle, P->outer_angle + h->S);
    h->joff.assign(h->S, 0.0);
    h->koff.assign(h->S, 0.0);
    if (P->j_offset) h->joff.assign(P->j_offset, P->j_offset + h->S);
    if (P->k_offset) h->koff.assign(P->k_offset, P->k_offset + h->S);
    h->seg0.assign(P->seg_start, P->seg_start + h->C);
    h->seg1.assign(P->seg_end, P->seg_end + h->C);
    h->geo_host.resize(h->S);
    for (int s = 0; s < h->S; ++s) {
        h->geo_host[s] = make_geom(h, s);
        h->xcopy = h->xcopy || h->geo_host[s].copy == 1;
    }
    if (prec != TT_F64) build_adj_params<float>(h, h->adj_f32);
    else build_adj_params<double>(h, h->adj_f64);

    const size_t es = h->esize();
#define ALLOC(ptr, bytes)                                                     \
    do {                                                                      \
        cudaError_t _e = cudaMalloc((void **)&(ptr), (bytes));                \
        if (_e != cudaSuccess) { free_handle(h); return cuda_fail(_e, "tt_create: cudaMalloc"); } \
    } while (0)
    ALLOC(h->geo, sizeof(ProjGeom) * h->S);
    ALLOC(h->B64, sizeof(double) * h->S * h->C * h->K);
    ALLOC(h->Bp, es * h->S * h->CP * h->KP);
    {
        const long long padded = (long long)(h->N[0] + 4) * (h->N[1] + 4) * (h->N[2] + 4);
        const long long copies = h->xcopy ? 2 : 1;
        h->pad_vox = padded;
        ALLOC(h->cpad, h->ssize() * copies * padded * h->KP);
        h->cpad_origin = 2LL * (h->N[1] + 4) * (h->N[2] + 4) + 2LL * (h->N[2] + 4) + 2;
        h->cpadx_origin = 2LL * (h->N[1] + 4) * (h->N[0] + 4) + 2LL * (h->N[0] + 4) + 2;
        cudaError_t ez = cudaMemsetAsync(h->cpad, 0, h->ssize() * copies * padded * h->KP, h->stream);   // border stays zero
        if (ez != cudaSuccess) { free_handle(h); return cuda_fail(ez, "tt_create: memset"); }
    }
    ALLOC(h->gpad, es * h->nvox() * h->KP);
    ALLOC(h->G, es * h->npix() * h->KP);
    plan_forward(h);
    h->fwd_staged = false;   // the tap-pair march is the faster one on every measured workload
    h->n_fwd_ctas = forward_ctas(h, h->fwd_staged);
    h->n_partials = std::max(forward_ctas(h, false), forward_ctas(h, true));
    ALLOC(h->partials, sizeof(double) * h->n_partials);
    ALLOC(h->loss_dev, sizeof(double) * 4);
    ALLOC(h->red, sizeof(double) * dot_blocks(h));
    {
        cudaError_t e = cudaMallocHost((void **)&h->loss_pinned, sizeof(double) * 4);
        if (e != cudaSuccess) { free_handle(h); return cuda_fail(e, "tt_create: cudaMallocHost"); }
        // the early-loss slot is optional: without a device mapping the loss
        // is read after the whole evaluation, as by every other entry point
        if (cudaHostAlloc((void **)&h->loss_slot_host, sizeof(LossSlot), cudaHostAllocMapped) == cudaSuccess) {
            h->loss_slot_host->value = 0.0;
            h->loss_slot_host->seq = 0;
            if (cudaHostGetDevicePointer((void **)&h->loss_slot_dev, h->loss_slot_host, 0) != cudaSuccess) {
                cudaFreeHost(h->loss_slot_host);
                h->loss_slot_host = h->loss_slot_dev = nullptr;
            }
        }
        (void)cudaGetLastError();
    }
    // basis matrix: stage [nodes][weights][frames 9S][seg0][seg1] and run the quadrature kernel
    std::vector<double> stage(2 * kQuadNodes + 9 * h->S + 2 * h->C);
    gauss_legendre(kQuadNodes, stage.data(), stage.data() + kQuadNodes);
    for (int s = 0; s < h->S; ++s) basis_frame(h->frame, h->inner[s], h->outer[s], stage.data() + 2 * kQuadNodes + 9 * s);
    std::memcpy(stage.data() + 2 * kQuadNodes + 9 * h->S, h->seg0.data(), sizeof(double) * h->C);
    std::memcpy(stage.data() + 2 * kQuadNodes + 9 * h->S + h->C, h->seg1.data(), sizeof(double) * h->C);
    double *dstage = nullptr;
    ALLOC(dstage, sizeof(double) * stage.size());
#undef ALLOC
    cudaError_t e = cudaMemcpyAsync(dstage, stage.data(), sizeof(double) * stage.size(), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->geo, h->geo_host.data(), sizeof(ProjGeom) * h->S, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = launch_basis(h, dstage, dstage + kQuadNodes);
    if (e == cudaSuccess) e = (prec != TT_F64) ? launch_cast_basis<float>(h) : launch_cast_basis<double>(h);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(dstage);
    if (e != cudaSuccess) {
        free_handle(h);
        return cuda_fail(e, "tt_create: basis set-up");
    }
    *out = h;
    return TT_OK;
}

tt_status tt_destroy(tt_handle *h)
{
    if (!h) return TT_OK;
    cudaStreamSynchronize(h->stream);
    free_handle(h);
    return TT_OK;
}

tt_status tt_set_stream(tt_handle *h, void *stream)
{
    if (!h) return invalid("null handle");
    const cudaStream_t next = (cudaStream_t)stream;
    if (next == h->stream) return TT_OK;
    // Order the new stream behind everything already enqueued on the old
    // one (no host synchronisation): the handle's scratch (G, partials,
    // the packed volume, the loss slot) may still be in use there.
    TT_CUDA(cudaEventRecord(h->stream_switch, h->stream), "tt_set_stream: event record");
    TT_CUDA(cudaStreamWaitEvent(next, h->stream_switch, 0), "tt_set_stream: stream wait");
    h->stream = next;
    return TT_OK;
}

tt_status tt_set_forward_kernel(tt_handle *h, int kind)
{
    if (!h) return invalid("null handle");
    if (kind < kFwdAuto || kind > kFwdStaged) return invalid("tt_set_forward_kernel: kind must be 0, 1 or 2");
    if (kind == kFwdStaged && h->stage_cap == 0) {
        set_error("tt_set_forward_kernel: the staged forward needs FP32 storage, 16 padded channels and a stage ring "
                  "that fits in shared memory");
        return TT_UNSUPPORTED;
    }
    h->fwd_staged = kind == kFwdStaged;
    h->n_fwd_ctas = forward_ctas(h, h->fwd_staged);
    return TT_OK;
}

tt_status tt_get_sizes(const tt_handle *h, int *K, int *KP, long long *n_vox, long long *n_data)
{
    if (!h) return invalid("null handle");
    if (K) *K = h->K;
    if (KP) *KP = h->KP;
    if (n_vox) *n_vox = h->nvox() * h->K;
    if (n_data) *n_data = h->ndata();
    return TT_OK;
}

tt_status tt_basis_matrix(tt_handle *h, double *B_dev)
{
    if (!h) return invalid("null handle");
    if (bad_ptr(B_dev)) return invalid("tt_basis_matrix: B_dev must be non-null and 16-byte aligned");
    TT_CUDA(cudaMemcpyAsync(B_dev, h->B64, sizeof(double) * h->S * h->C * h->K, cudaMemcpyDeviceToDevice, h->stream),
            "basis copy");
    return TT_OK;
}

tt_status tt_project(tt_handle *h, const float *c, float *I)
{
    tt_status st = check_handle(h, TT_F32);
    return st != TT_OK ? st : project_impl<float>(h, c, I);
}

tt_status tt_project_f64(tt_handle *h, const double *c, double *I)
{
    tt_status st = check_handle(h, TT_F64);
    return st != TT_OK ? st : project_impl<double>(h, c, I);
}

tt_status tt_adjoint(tt_handle *h, const float *R, float *g)
{
    tt_status st = check_handle(h, TT_F32);
    return st != TT_OK ? st : adjoint_impl<float>(h, R, g);
}

tt_status tt_adjoint_f64(tt_handle *h, const double *R, double *g)
{
    tt_status st = check_handle(h, TT_F64);
    return st != TT_OK ? st : adjoint_impl<double>(h, R, g);
}

tt_status tt_gradient_residual(tt_handle *h, const float *c, const float *I, const float *W, float *g,
                               double *loss_host)
{
    tt_status st = check_handle(h, TT_F32);
    return st != TT_OK ? st : grad_impl<float>(h, c, I, W, g, loss_host);
}

tt_status tt_gradient_residual_f64(tt_handle *h, const double *c, const double *I, const double *W, double *g,
                                   double *loss_host)
{
    tt_status st = check_handle(h, TT_F64);
    return st != TT_OK ? st : grad_impl<double>(h, c, I, W, g, loss_host);
}

// Device address of page-locked, device-mapped host memory (the device can
// load and store it directly over the host link), else NULL.
static const void *mapped_device_pointer(const void *host)
{
    cudaPointerAttributes pa;
    if (host && cudaPointerGetAttributes(&pa, host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer)
        return pa.devicePointer;
    cudaGetLastError();   // clear the query's error state for unregistered memory
    return nullptr;
}

tt_status tt_gradient_residual_host(tt_handle *h, const float *c_host, const float *I_host, const float *W_host,
                                    float *g_host, double *loss_host)
{
    tt_status st = check_handle(h, TT_F32);
    if (st != TT_OK) return st;
    if (!c_host || !I_host || !g_host || !loss_host)
        return invalid("tt_gradient_residual_host: c, I, g, loss must not be NULL");
    const size_t bc = sizeof(float) * h->nvox() * h->K, bd = sizeof(float) * h->ndata();
    // Inputs go through device staging buffers: c first on the compute
    // stream, then I and W in Q projection chunks on a copy stream.  The
    // forward launch of chunk q waits only for chunk q and runs on one of two
    // side streams, so that a chunk's last wave overlaps the next chunk's
    // first; the adjoint joins both.  (Reading mapped inputs in place over
    // the host link measured slower than these copies.)
    // A page-locked, device-mapped g_host is written by the adjoint in place,
    // its stores crossing the host link while the kernel runs; any other
    // g_host gets the gradient with one copy.
    float *g_map = (float *)mapped_device_pointer(g_host);
    const int Q = std::min(8, h->S);
    if (!h->hc) TT_CUDA(cudaMalloc(&h->hc, bc), "host-path cudaMalloc");
    if (!g_map && !h->hg) TT_CUDA(cudaMalloc(&h->hg, bc), "host-path cudaMalloc");
    if (!h->hI) TT_CUDA(cudaMalloc(&h->hI, bd), "host-path cudaMalloc");
    if (W_host && !h->hW) TT_CUDA(cudaMalloc(&h->hW, bd), "host-path cudaMalloc");
    if (!h->copy_stream) TT_CUDA(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (cudaStream_t &t : h->side)
        if (!t) TT_CUDA(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking), "side stream");
    while ((int)h->chunk_ready.size() < Q + 4) {
        cudaEvent_t e;
        TT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "chunk event");
        h->chunk_ready.push_back(e);
    }
    TT_CUDA(cudaMemcpyAsync(h->hc, c_host, bc, cudaMemcpyHostToDevice, h->stream), "H2D c");
    TT_CUDA(cudaEventRecord(h->chunk_ready[Q], h->stream), "event");
    TT_CUDA(cudaStreamWaitEvent(h->copy_stream, h->chunk_ready[Q], 0), "stream wait");
    const size_t per_proj = (size_t)h->nj * h->nk * h->C;
    for (int q = 0; q < Q; ++q) {
        const int s0 = (int)((long long)h->S * q / Q), s1 = (int)((long long)h->S * (q + 1) / Q);
        const size_t off = per_proj * s0, n = per_proj * (s1 - s0);
        TT_CUDA(cudaMemcpyAsync((float *)h->hI + off, I_host + off, sizeof(float) * n, cudaMemcpyHostToDevice,
                                h->copy_stream), "H2D I");
        if (W_host)
            TT_CUDA(cudaMemcpyAsync((float *)h->hW + off, W_host + off, sizeof(float) * n, cudaMemcpyHostToDevice,
                                    h->copy_stream), "H2D W");
        TT_CUDA(cudaEventRecord(h->chunk_ready[q], h->copy_stream), "event");
    }
    const float *I = (const float *)h->hI, *W = W_host ? (const float *)h->hW : nullptr;
    cudaEvent_t packed = h->chunk_ready[Q + 1], side_done[2] = {h->chunk_ready[Q + 2], h->chunk_ready[Q + 3]};
    const cudaStream_t main_stream = h->stream;
    st = with_storage<float>(h, [&]<typename S>() -> tt_status {
        TT_CUDA((launch_pack<float, S>(h, (const float *)h->hc)), "pack");
        TT_CUDA(cudaEventRecord(packed, main_stream), "event");
        for (int t = 0; t < 2; ++t) TT_CUDA(cudaStreamWaitEvent(h->side[t], packed, 0), "stream wait");
        cudaError_t e = cudaSuccess;
        for (int q = 0; q < Q && e == cudaSuccess; ++q) {
            const int s0 = (int)((long long)h->S * q / Q), s1 = (int)((long long)h->S * (q + 1) / Q);
            e = cudaStreamWaitEvent(h->side[q & 1], h->chunk_ready[q], 0);
            h->stream = h->side[q & 1];          // the launcher enqueues on h->stream
            if (e == cudaSuccess) e = launch_forward<float, S>(h, nullptr, I, W, true, s0, s1);
            h->stream = main_stream;
        }
        TT_CUDA(e, "forward");
        for (int t = 0; t < 2; ++t) {
            TT_CUDA(cudaEventRecord(side_done[t], h->side[t]), "event");
            TT_CUDA(cudaStreamWaitEvent(main_stream, side_done[t], 0), "stream wait");
        }
        TT_CUDA((launch_adjoint<float, S>(h, g_map ? g_map : (float *)h->hg, true)), "adjoint");
        return TT_OK;
    });
    if (st != TT_OK) return st;
    if (!g_map) TT_CUDA(cudaMemcpyAsync(g_host, h->hg, bc, cudaMemcpyDeviceToHost, h->stream), "D2H g");
    return tt_read_loss(h, loss_host);
}

tt_status tt_profile_enable(tt_handle *h, int enable)
{
    if (!h) return invalid("null handle");
    h->prof.enabled = enable != 0;
    while (h->prof.enabled && h->prof.free_events.size() + 2 * h->prof.pending.size() < kProfileEvents) {
        cudaEvent_t e;
        TT_CUDA(cudaEventCreate(&e), "event create");
        h->prof.free_events.push_back(e);
    }
    return TT_OK;
}

tt_status tt_profile_reset(tt_handle *h)
{
    if (!h) return invalid("null handle");
    TT_CUDA(cudaStreamSynchronize(h->stream), "stream synchronize");
    for (const auto &r : h->prof.pending) {
        h->prof.free_events.push_back(r.begin);
        if (r.free_end) h->prof.free_events.push_back(r.end);
    }
    h->prof.pending.clear();
    for (int i = 0; i < TT_KSLOT_COUNT; ++i) { h->prof.total_ms[i] = 0.0; h->prof.launches[i] = 0; }
    return TT_OK;
}

tt_status tt_profile_read(tt_handle *h, int slot, double *total_ms, long long *launches)
{
    if (!h) return invalid("null handle");
    if (slot < 0 || slot >= TT_KSLOT_COUNT) return invalid("bad kernel slot");
    TT_CUDA(prof_fold(h, true, (size_t)-1), "profile events");
    if (total_ms) *total_ms = h->prof.total_ms[slot];
    if (launches) *launches = h->prof.launches[slot];
    return TT_OK;
}

const char *tt_kernel_slot_name(int slot)
{
    static const char *names[TT_KSLOT_COUNT] = {"pack", "forward", "backcontract", "adjoint",
                                                "unpack", "reduce", "basis", "vector"};
    return (slot >= 0 && slot < TT_KSLOT_COUNT) ? names[slot] : "";
}

long long tt_launch_count(const tt_handle *h) { return h ? h->launch_count : 0; }

}  // extern "C"
