// tt_noalloc.cu -- tt_basis_matrix_noalloc: the basis-matrix quadrature for
// callers that cannot allocate device memory.  Its scratch (Gauss-Legendre
// nodes and weights, the rotated frame of every projection, the segment
// bounds) lives in a fixed file-scope device array instead of a cudaMalloc'd
// buffer.
#include <cmath>
#include <mutex>

#include "tt_internal.cuh"

namespace tt {

// k_basis is the quadrature kernel of tt_create (tt_misc.cu).
__global__ void k_basis(const double *__restrict__ frames, const double *__restrict__ seg0,
                        const double *__restrict__ seg1, const double *__restrict__ nodes,
                        const double *__restrict__ weights, double cth, double sth, int L, int K, int C,
                        double *__restrict__ B);

constexpr int kNoAllocMaxProj = 2048;
constexpr int kNoAllocDoubles = 2 * kQuadNodes + 9 * kNoAllocMaxProj + 2 * kMaxSeg;   // 18,624 doubles, 145.5 KiB

// Scratch of tt_basis_matrix_noalloc, resident on every device that loads
// libtt until the process exits.  Layout: nodes[32], weights[32],
// frames[n_proj][9] (p_s, q0_s, q90_s), seg_start[n_seg], seg_end[n_seg].
static __device__ __align__(256) double g_basis_scratch[kNoAllocDoubles];

static std::mutex g_scratch_mu;
static double *g_scratch_addr[256];          // device address of g_basis_scratch, per device ordinal

static thread_local double t_host_stage[kNoAllocDoubles];

static void rodrigues(const double *n_in, double t, double R[9])
{
    const double nn = std::sqrt(n_in[0] * n_in[0] + n_in[1] * n_in[1] + n_in[2] * n_in[2]);
    const double x = n_in[0] / nn, y = n_in[1] / nn, z = n_in[2] / nn;
    const double c = std::cos(t), s = std::sin(t), C1 = 1.0 - c;
    R[0] = c + x * x * C1;     R[1] = x * y * C1 - z * s; R[2] = x * z * C1 + y * s;
    R[3] = y * x * C1 + z * s; R[4] = c + y * y * C1;     R[5] = y * z * C1 - x * s;
    R[6] = z * x * C1 - y * s; R[7] = z * y * C1 + x * s; R[8] = c + z * z * C1;
}

}  // namespace tt

extern "C" tt_status tt_basis_matrix_noalloc(const tt_problem *prob, double *B_dev, void *stream)
{
    using namespace tt;
    tt_status st = validate(prob);
    if (st != TT_OK) return st;
    if (prob->ell_max > kMaxEll) {
        set_error("tt_basis_matrix_noalloc: ell_max above 12 has no compiled kernels");
        return TT_UNSUPPORTED;
    }
    if (prob->n_proj > kNoAllocMaxProj) {
        set_error("tt_basis_matrix_noalloc: n_proj exceeds the fixed scratch capacity of 2048 projections");
        return TT_INVALID_ARG;
    }
    if (B_dev == nullptr || (reinterpret_cast<uintptr_t>(B_dev) & 15u) != 0) {
        set_error("tt_basis_matrix_noalloc: B_dev must be non-null and 16-byte aligned");
        return TT_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "tt_basis_matrix_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 256) {
        set_error("tt_basis_matrix_noalloc: device ordinal out of range");
        return TT_UNSUPPORTED;
    }
    double *scratch = nullptr;
    {
        // One-time set-up per device (the device is current here): the host
        // name g_basis_scratch is only a stand-in, the kernel needs the
        // device address.
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_basis_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "tt_basis_matrix_noalloc: cudaGetSymbolAddress");
            g_scratch_addr[dev] = static_cast<double *>(p);
        }
        scratch = g_scratch_addr[dev];
    }

    // Stage the quadrature rule, the rotated frames and the segments on the host.
    const int S = prob->n_proj, C = prob->n_seg, L = prob->ell_max, K = (L + 1) * (L + 2) / 2;
    double *hs = t_host_stage;
    gauss_legendre(kQuadNodes, hs, hs + kQuadNodes);
    for (int s = 0; s < S; ++s) {
        double Ra[9], Rb[9], R[9];
        rodrigues(prob->frame.inner_axis, prob->inner_angle[s], Ra);
        rodrigues(prob->frame.outer_axis, prob->outer_angle[s], Rb);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) R[3 * r + c] = Rb[3 * r] * Ra[c] + Rb[3 * r + 1] * Ra[3 + c] + Rb[3 * r + 2] * Ra[6 + c];
        const double *vecs[3] = {prob->frame.p, prob->frame.q0, prob->frame.q90};
        double *F = hs + 2 * kQuadNodes + 9 * s;
        for (int t = 0; t < 3; ++t)
            for (int c = 0; c < 3; ++c)       // R_s^T v
                F[3 * t + c] = R[c] * vecs[t][0] + R[3 + c] * vecs[t][1] + R[6 + c] * vecs[t][2];
    }
    double *seg0 = hs + 2 * kQuadNodes + 9 * S, *seg1 = seg0 + C;
    for (int c = 0; c < C; ++c) { seg0[c] = prob->seg_start[c]; seg1[c] = prob->seg_end[c]; }
    const size_t n = (size_t)(2 * kQuadNodes + 9 * S + 2 * C);

    cudaStream_t strm = (cudaStream_t)stream;
    e = cudaMemcpyAsync(scratch, hs, n * sizeof(double), cudaMemcpyHostToDevice, strm);
    if (e != cudaSuccess) return cuda_fail(e, "tt_basis_matrix_noalloc: staging copy");
    const double th = 0.5 * prob->two_theta;
    const double *frames = scratch + 2 * kQuadNodes;
    k_basis<<<dim3(C, S), kQuadNodes, kQuadNodes * K * sizeof(double), strm>>>(
        frames, frames + 9 * S, frames + 9 * S + C, scratch, scratch + kQuadNodes, std::cos(th), std::sin(th), L, K,
        C, B_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tt_basis_matrix_noalloc: launch");
    return TT_OK;
}
