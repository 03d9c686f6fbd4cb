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
    // the same frames as tt_create stages (one shared helper)
    for (int s = 0; s < S; ++s) basis_frame(prob->frame, prob->inner_angle[s], prob->outer_angle[s], hs + 2 * kQuadNodes + 9 * s);
    double *seg0 = hs + 2 * kQuadNodes + 9 * S, *seg1 = seg0 + C;
    for (int c = 0; c < C; ++c) { seg0[c] = prob->seg_start[c]; seg1[c] = prob->seg_end[c]; }
    const size_t n = (size_t)(2 * kQuadNodes + 9 * S + 2 * C);

    cudaStream_t strm = (cudaStream_t)stream;
    // A copy from pageable host memory: the runtime waits for the work
    // already on strm, then stages the bytes before this call returns, so
    // the thread's staging buffer may be reused by its next call.
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
