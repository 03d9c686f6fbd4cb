// tt_conv.cu -- 3x3x3 convolutions of the learned warm start on the tensor
// cores (bfloat16 inputs, float accumulation): the forward convolution (and
// with flipped weights the data gradient) on tcgen05 with tensor-memory
// accumulators, the weight gradient with mma.sync m16n8k16; and the small
// kernels of the training step (ReLU mask, squared error, Adam).
//
// Layouts: activations a[v][C] bfloat16, v = (x*ny + y)*nz + z, C in {16, 32}
// (channels zero padded); convolution weights wk[t][Cout][Cin] bfloat16, t =
// (dx+1)*9 + (dy+1)*3 + (dz+1); "same" zero padding, cross-correlation:
//   y[v][co] = sum_t sum_ci a[v + d_t][ci] * wk[t][co][ci].
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "tt_internal.cuh"
#include "tt_umma.cuh"

namespace tt {

// ------------------------------------------------------------ mma helpers

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void *smem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned (&r)[4], const void *smem)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// D = A (16x16 bf16, row) * B (16x8 bf16, col) + D, float accumulators.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// ------------------------------------------------ forward conv, tcgen05
//
// Implicit GEMM on the fifth-generation tensor cores.  A tile covers one x
// plane, four y rows and a window of 32 input z (z0-1 .. z0+30) whose inner
// 30 are the tile's output z.  For each of the 9 in-plane tap offsets
// (dx, dy) one MMA chain multiplies the 128 input rows (row m = 32 y + z,
// 16 bytes apart, so a y offset is a change of descriptor start address and
// an x offset another staged plane) by the three z taps' weights stacked as
// N = 3 COUT columns:
//   P_dz[row][co] = sum_{dx,dy,ci} x[x0+dx-1][y+dy-1][row z][ci] w[(dx,dy,dz)][co][ci]
// and the epilogue applies the z taps by shifting rows between lanes:
//   y(z) = P_0(z - 1) + P_1(z) + P_2(z + 1).
// That is 9 * CIN / 16 MMAs of M 128, N 3 COUT, K 16 per tile, a third of
// the count with the z taps as separate MMAs of N COUT; the MMA chain, not
// the N width, sets the time at these sizes.  Plane buffers are [CIN/8][y 6]
// [z 32] 16-byte (8-channel) chunks, zeros outside the volume: SBO = 128 B
// (next 8 rows), LBO = 6 * 512 B (next 8 channels).  Weights are staged once
// per CTA as [dx,dy][CIN/8][dz * COUT + co][8] (SBO = 128 B, LBO = 3 COUT
// 16 B).
//
// Pipeline.  A persistent CTA walks runs of consecutive x planes of one (y, z)
// tile column.  Tile x needs planes x-1, x, x+1 from a ring of NBUF plane
// buffers (4 for 32 -> 32 channels, more where the weights are smaller), so
// each step stages one new plane, NBUF - 3 steps ahead.  A plane is one tiled tensor
// copy: the input viewed as a 5-D tensor (8 channels, z, y, channel group,
// x) whose box of 8 x 32 x 6 x CIN/8 x 1 elements lands in exactly the
// buffer layout above, zeros outside the volume; it completes on the
// buffer's own mbarrier.  Step for tile x: thread 0 waits for plane x+1's
// copy, issues the tile's MMAs into tensor-memory accumulator x % 2 and
// commits them to mbarrier x % 2; meanwhile all eight warps wait for tile
// x-1's mbarrier, thread 0 starts the copy of plane x-2+NBUF into the buffer
// that tile x-1 was the last to read, and all write tile x-1 out (ReLU, bf16
// or f32).  (Staging the planes through registers by all warps was
// measured 0.162 ms for the 32 -> 32 layer at 128^3.)  A wait that gives up
// writes NaN into its tile, which every consumer of the output sees; at exit
// thread 0 waits (bounded) for copies still in flight.
constexpr uint32_t kTcWaitTries = 1u << 22;
constexpr int kTcThreads = 256;
constexpr int kTileZ = 30;                 // output z per tile (32 input rows)

template <int CIN, int COUT>
struct TcConvSmem {
    static constexpr uint32_t plane = (CIN / 8) * 6 * 512;
    static constexpr uint32_t dxy = 3 * COUT * CIN * 2;       // weights of one (dx, dy): three z taps
    // plane buffers: as many as leave two CTAs per SM (110 KB each), 4..8
    static constexpr int nbuf_fit = (int)((110u * 1024u - 9 * dxy - 256) / plane);
    static constexpr int nbuf = nbuf_fit > 8 ? 8 : (nbuf_fit < 4 ? 4 : nbuf_fit);
    static constexpr uint32_t wts = nbuf * plane;
    // [0, 1] MMA commits, [2, 2 + nbuf) plane copies, then the tensor-memory
    // slot and a failure flag
    static constexpr uint32_t mbar = wts + 9 * dxy;
    static constexpr uint32_t bytes = mbar + 8 * (2 + nbuf) + 8;
    static constexpr uint32_t tmem_cols = 2 * 3 * COUT <= 128 ? 128 : 256;   // two accumulators of 3 COUT
};

// Tile epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. (input rows
// y0 + w % 4, z0 - 1 + lane) and, for its half of the output channels, the
// three z-tap blocks of accumulator `acc_col`; lanes 1..30 combine rows
// lane-1, lane, lane+1 and write output z0 - 1 + lane.
template <int COUT, bool RELU, bool OUT_F32>
__device__ __forceinline__ void tile_epilogue(uint32_t tmem, uint32_t acc_col, bool ok, void *__restrict__ out, int x0,
                                              int y0, int z0, int ny, int nz, int warp, int lane)
{
    constexpr int CW = COUT / (kTcThreads / 128);
    static_assert(CW == 8 || CW == 16, "a warp reads 8 or 16 accumulator columns per z tap");
    const int quad = warp & 3, c_base = (warp >> 2) * CW;
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    float p[3][CW];
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
        const uint32_t taddr = tmem + lanes + acc_col + (uint32_t)(dz * COUT + c_base);
        if constexpr (CW == 16) umma::tmem_ld16(taddr, p[dz]);
        else umma::tmem_ld8(taddr, p[dz]);
    }
    float v[CW];
#pragma unroll
    for (int c = 0; c < CW; ++c) {
        const float below = __shfl_up_sync(0xffffffffu, p[0][c], 1);      // P_0 of row lane-1
        const float above = __shfl_down_sync(0xffffffffu, p[2][c], 1);     // P_2 of row lane+1
        v[c] = ok ? (below + p[1][c]) + above : __int_as_float(0x7fc00000);
    }
    const int gy = y0 + quad, gz = z0 - 1 + lane;
    if (lane < 1 || lane > kTileZ || gy >= ny || gz >= nz) return;
    const size_t vox = ((size_t)x0 * ny + gy) * nz + gz;
    if constexpr (OUT_F32) {
        float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(out) + vox * COUT + c_base);
#pragma unroll
        for (int i = 0; i < CW / 4; ++i) {
            float4 q = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            if (RELU) { q.x = fmaxf(q.x, 0.f); q.y = fmaxf(q.y, 0.f); q.z = fmaxf(q.z, 0.f); q.w = fmaxf(q.w, 0.f); }
            o[i] = q;
        }
    } else {
        uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(out) + vox * COUT + c_base);
#pragma unroll
        for (int i = 0; i < CW / 8; ++i) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float a = v[8 * i + 2 * j], b = v[8 * i + 2 * j + 1];
                if (RELU) { a = fmaxf(a, 0.f); b = fmaxf(b, 0.f); }
                const __nv_bfloat162 h2 = __floats2bfloat162_rn(a, b);
                w[j] = *reinterpret_cast<const uint32_t *>(&h2);
            }
            o[i] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

template <int CIN, int COUT, bool RELU, bool OUT_F32>
__global__ void __launch_bounds__(kTcThreads)
k_conv3d_fwd_tc(const __grid_constant__ CUtensorMap planes, const __nv_bfloat16 *__restrict__ wk,
                void *__restrict__ out, int nx, int ny, int nz, int tiles_y, int tiles_z)
{
    using L = TcConvSmem<CIN, COUT>;
    constexpr int KC = CIN / 8, NB = 3 * COUT;
    constexpr uint32_t kLboA = 6 * 512, kLboB = NB * 16;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + L::mbar);   // [0, 1] MMA commits
    constexpr int NBUF = L::nbuf;
    uint64_t *pbar = mbar + 2;                                        // [NBUF] plane copies, one per buffer
    uint32_t *tslot = reinterpret_cast<uint32_t *>(pbar + NBUF);
    volatile int &s_fail = *reinterpret_cast<volatile int *>(tslot + 1);   // a plane copy not seen landing
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) umma::tmem_alloc(tslot, L::tmem_cols);
    if (tid == 0) {
        for (int i = 0; i < 2 + NBUF; ++i) umma::mbar_init(mbar + i, 1);
        s_fail = 0;
    }
    // weights [t][co][ci], t = 9 dx + 3 dy + dz  ->  [dx,dy][ci/8][dz COUT + co][8]
    for (int e = tid; e < 27 * COUT * KC; e += kTcThreads) {
        const int kc = e % KC, co = (e / KC) % COUT, t = e / (KC * COUT);
        const int dxy = t / 3, dz = t % 3;
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(wk + ((size_t)t * COUT + co) * CIN) + kc);
        *reinterpret_cast<uint4 *>(smem + L::wts + dxy * L::dxy + kc * kLboB + (dz * COUT + co) * 16) = v;
    }
    umma::fence_async_smem();
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = umma::idesc_bf16_f32(128, NB);
    const uint32_t s_planes = umma::smem_u32(smem), s_wts = umma::smem_u32(smem + L::wts);
    // Phase parities as bit masks (bit b for mbarrier b): the next wait on
    // each MMA mbarrier; on each plane buffer (thread 0) the next wait, the
    // count of copies started mod 2, and whether any was started.
    uint32_t mma_par = 0, wait_par = 0, copy_par = 0, used = 0;
    const void *pmap = &planes;

    // This CTA's equal share [t_begin, t_end) of the tile sequence (x fastest,
    // then the z tile, then the y tile), walked as runs of consecutive x.
    const long long n_tiles = (long long)nx * tiles_y * tiles_z;
    const long long t_begin = n_tiles * blockIdx.x / gridDim.x, t_end = n_tiles * (blockIdx.x + 1) / gridDim.x;
    for (long long t = t_begin; t < t_end;) {
        const long long col = t / nx;
        const int tz = (int)(col % tiles_z), ty = (int)(col / tiles_z);
        const int y0 = ty * 4, z0 = tz * kTileZ, xa = (int)(t - col * nx);
        const int xb = (int)std::min<long long>(nx, xa + (t_end - t));
        t += xb - xa;
        // thread 0 starts and awaits the copies; plane px (>= -1) goes to
        // buffer (px + NBUF) % NBUF
        auto copy_plane = [&](int px) {
            const int bf = (px + NBUF) % NBUF;
            umma::mbar_arrive_expect_tx(pbar + bf, L::plane);
            umma::tma_load_5d(smem + bf * L::plane, pmap, 0, z0 - 1, y0 - 1, 0, px, pbar + bf);
            copy_par ^= 1u << bf;
            used |= 1u << bf;
        };
        auto await_plane = [&](int px) {
            const int bf = (px + NBUF) % NBUF;
            if (!umma::mbar_wait(pbar + bf, (wait_par >> bf) & 1u, kTcWaitTries)) s_fail = 1;
            wait_par ^= 1u << bf;
        };
        // planes xa-1 .. xa+NBUF-2 (the ring is idle here: the previous run's MMAs are done)
        if (tid == 0)
            for (int px = xa - 1; px <= xa + NBUF - 2 && px <= xb; ++px) copy_plane(px);
        for (int x = xa; x <= xb; ++x) {
            const int i = x - xa;                 // step: tile x issued, tile x-1 written out, plane x+2 started
            umma::fence_before_sync();
            __syncthreads();
            umma::fence_after_sync();
            if (x < xb && tid == 0) {
                if (i == 0) { await_plane(x - 1); await_plane(x); }
                await_plane(x + 1);
                const uint32_t acc = tmem + (uint32_t)(NB * (i & 1));
                for (int dxy = 0; dxy < 9; ++dxy) {
                    const int dx = dxy / 3, dy = dxy % 3;                  // offset + 1
                    const uint32_t a0 = s_planes + ((x - 1 + dx + NBUF) % NBUF) * L::plane + dy * 512;
                    const uint32_t b0 = s_wts + dxy * L::dxy;
#pragma unroll
                    for (int kk = 0; kk < CIN / 16; ++kk)
                        umma::mma_bf16(acc, umma::smem_desc(a0 + kk * 2 * kLboA, kLboA, 128),
                                       umma::smem_desc(b0 + kk * 2 * kLboB, kLboB, 128), idesc, (dxy | kk) ? 1u : 0u);
                }
                umma::mma_commit(mbar + (i & 1));
            }
            if (i > 0) {
                const int p = (i - 1) & 1;
                const bool ok = umma::mbar_wait(mbar + p, (mma_par >> p) & 1u, kTcWaitTries) && !s_fail;
                mma_par ^= 1u << p;
                // tile x-1, the last reader of plane x-2's buffer, is done: that
                // buffer takes plane x-2+NBUF now, before the tile is written out
                if (tid == 0 && x - 2 + NBUF <= xb) copy_plane(x - 2 + NBUF);
                umma::fence_after_sync();
                tile_epilogue<COUT, RELU, OUT_F32>(tmem, (uint32_t)(NB * p), ok, out, x - 1, y0, z0, ny, nz, warp,
                                                   lane);
            }
        }
        umma::fence_before_sync();
        __syncthreads();                       // ring and accumulators free for the next run
        umma::fence_after_sync();
    }
    // after a wait that gave up, a copy may still be writing shared memory:
    // wait (bounded) for the last copy into every buffer
    if (tid == 0 && s_fail)
        for (int bf = 0; bf < NBUF; ++bf)
            if ((used >> bf) & 1u) umma::mbar_wait(pbar + bf, ((copy_par >> bf) & 1u) ^ 1u, kTcWaitTries);
    if (warp == 0) umma::tmem_dealloc(tmem, L::tmem_cols);
}

// ------------------------------------------------------- weight gradient
//
// dw[t][co][ci] += sum_v dy[v][co] * x[v + d_t][ci]  (float, atomics per CTA).
// CTA = one tap (blockIdx.y) x a strided share of the 16-voxel z segments;
// each warp stages its segment of dy and of the shifted x in its own shared
// rows and multiplies dy^T (co x v) by x (v x ci) with transposing ldmatrix.
template <int CIN, int COUT>
__global__ void __launch_bounds__(256)
k_conv3d_wgrad(const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ dy, float *__restrict__ dw,
               int nx, int ny, int nz)
{
    constexpr int RX = CIN + 8, RY = COUT + 8;
    __shared__ __align__(16) __nv_bfloat16 sx[8][16 * RX];
    __shared__ __align__(16) __nv_bfloat16 sy[8][16 * RY];
    __shared__ float red[COUT * CIN];

    const int t = blockIdx.y;
    const int dx = t / 9 - 1, dyy = (t / 3) % 3 - 1, dz = t % 3 - 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int zsegs = (nz + 15) / 16;
    const long long nseg = (long long)nx * ny * zsegs;
    constexpr int MT = COUT / 16, NT = CIN / 8;
    float acc[MT][NT][4];
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int i = 0; i < 4; ++i) acc[m][n][i] = 0.f;

    for (long long sg = (long long)blockIdx.x * 8 + warp; sg < nseg; sg += (long long)gridDim.x * 8) {
        const int zs = (int)(sg % zsegs), yv = (int)((sg / zsegs) % ny), xv = (int)(sg / ((long long)zsegs * ny));
        // stage 16 rows of dy (zeros past nz) and of x shifted by the tap
        for (int e = lane; e < 16 * (COUT / 8); e += 32) {
            const int r = e / (COUT / 8), c = e % (COUT / 8);
            const int zv = zs * 16 + r;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (zv < nz) v = __ldg(reinterpret_cast<const uint4 *>(dy + (((long long)xv * ny + yv) * nz + zv) * COUT) + c);
            *reinterpret_cast<uint4 *>(&sy[warp][r * RY + c * 8]) = v;
        }
        for (int e = lane; e < 16 * (CIN / 8); e += 32) {
            const int r = e / (CIN / 8), c = e % (CIN / 8);
            const int zv = zs * 16 + r;
            const int gx = xv + dx, gy = yv + dyy, gz = zv + dz;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (zv < nz && (unsigned)gx < (unsigned)nx && (unsigned)gy < (unsigned)ny && (unsigned)gz < (unsigned)nz)
                v = __ldg(reinterpret_cast<const uint4 *>(x + (((long long)gx * ny + gy) * nz + gz) * CIN) + c);
            *reinterpret_cast<uint4 *>(&sx[warp][r * RX + c * 8]) = v;
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            unsigned a[4];
            ldsm_x4_t(a, &sy[warp][((lane >> 4) * 8 + (lane & 7)) * RY + 16 * m + ((lane >> 3) & 1) * 8]);
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                unsigned bb[4];
                ldsm_x4_t(bb, &sx[warp][(((lane >> 3) & 1) * 8 + (lane & 7)) * RX + 16 * np + (lane >> 4) * 8]);
                mma_bf16(acc[m][2 * np], a, bb[0], bb[1]);
                mma_bf16(acc[m][2 * np + 1], a, bb[2], bb[3]);
            }
        }
        __syncwarp();
    }

    // CTA reduction of the 8 warps' partial sums, then one atomic per element
    for (int i = threadIdx.x; i < COUT * CIN; i += blockDim.x) red[i] = 0.f;
    __syncthreads();
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int m = 0; m < MT; ++m)
#pragma unroll
        for (int n = 0; n < NT; ++n)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int co = 16 * m + g + 8 * (i >> 1), ci = 8 * n + 2 * tig + (i & 1);
                atomicAdd(&red[co * CIN + ci], acc[m][n][i]);
            }
    __syncthreads();
    for (int i = threadIdx.x; i < COUT * CIN; i += blockDim.x) atomicAdd(&dw[(long long)t * COUT * CIN + i], red[i]);
}

// ------------------------------------------------------------ small kernels

// d[i] = a[i] > 0 ? d[i] : 0 (ReLU backward, in place), bfloat16.
__global__ void k_relu_mask(const __nv_bfloat16 *__restrict__ a, __nv_bfloat16 *__restrict__ d, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!(__bfloat162float(a[i]) > 0.f)) d[i] = __float2bfloat16(0.f);
}

// Squared error of y [nvox][16] (float, channels >= k_real ignored) against
// tgt_scale * target [nvox][k_real]: partial sums of (y - t)^2 (FP64) and, if
// dy, dy[v][c] = 2 (y - t) * inv_count (bfloat16, zero on padded channels).
__global__ void k_sq_error(const float *__restrict__ y, const float *__restrict__ tgt, float tgt_scale, int k_real,
                           long long nvox, double inv_count, __nv_bfloat16 *__restrict__ dy,
                           double *__restrict__ partials)
{
    __shared__ double red[32];
    double s = 0.0;
    const long long n = nvox * 16;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i >> 4;
        const int c = (int)(i & 15);
        float d = 0.f;
        if (c < k_real) {
            d = y[i] - tgt_scale * tgt[v * k_real + c];
            s += (double)d * d;
        }
        if (dy) dy[i] = __float2bfloat16((float)(2.0 * inv_count) * d);
    }
    __syncthreads();
    double v = s;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) u += __shfl_down_sync(0xffffffffu, u, off);
        if (threadIdx.x == 0) partials[blockIdx.x] = u;
    }
}

// x [nvox][k_real] float -> a [nvox][16] bfloat16, scaled, zero padded.
__global__ void k_pack_bf16(const float *__restrict__ x, int k_real, long long nvox, float scale,
                            __nv_bfloat16 *__restrict__ a)
{
    const long long n = nvox * 16;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i >> 4;
        const int c = (int)(i & 15);
        a[i] = __float2bfloat16(c < k_real ? scale * x[v * k_real + c] : 0.f);
    }
}

// y [nvox][16] float -> out [nvox][k_real], scaled.
__global__ void k_unpack_f32(const float *__restrict__ y, int k_real, long long nvox, float scale, float *__restrict__ out)
{
    const long long n = nvox * k_real;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long v = i / k_real;
        const int c = (int)(i - v * k_real);
        out[i] = scale * y[v * 16 + c];
    }
}

// Master weights w [27][R][Cc] (float, padded) -> wk bfloat16, either the same
// layout (flip = 0) or that of the transposed convolution (flip = 1):
// wk[t][c][r] = w[26 - t][r][c].
__global__ void k_cast_conv_weights(const float *__restrict__ w, int R, int Cc, int flip, __nv_bfloat16 *__restrict__ wk)
{
    const int n = 27 * R * Cc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float v;
        if (!flip) {
            v = w[i];
        } else {
            const int r = i % R, c = (i / R) % Cc, t = i / (R * Cc);   // output [t][c][r]
            v = w[((26 - t) * R + r) * Cc + c];
        }
        wk[i] = __float2bfloat16(v);
    }
}

// Adam (Kingma & Ba) on float parameters with bias-corrected moments.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

static int sm_count() { return current_sm_count(); }

static unsigned grid_n(long long n)
{
    const long long cap = 16LL * sm_count();
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// Launches the forward convolution (tcgen05 kernel) for a (CIN, COUT) pair:
// persistent CTAs (two per SM when the staging fits), each walking an equal
// contiguous share of the nx * tiles_y * tiles_z tiles (x fastest) as runs
// of consecutive x planes (measured at 128^3, 32 -> 32 channels: runs of 16
// planes dealt round robin left a 19% tail; equal shares cut it and the
// pipeline fills to about 1.5 runs per CTA).
cudaError_t conv3d_forward(const __nv_bfloat16 *in, const __nv_bfloat16 *wk, void *out, int nx, int ny, int nz, int cin,
                           int cout, bool relu, bool out_f32, cudaStream_t st)
{
    const int tiles_y = (ny + 3) / 4, tiles_z = (nz + kTileZ - 1) / kTileZ;
    if (nx < 1 || ny < 1 || nz < 1) return cudaSuccess;
    if (cin != 16 && cin != 32) return cudaErrorInvalidValue;
    // Input planes: the activations [x][y][z][cin] viewed as the 5-D tensor
    // (8 channels, z, y, channel group, x) -- strides 2, 2 cin, 2 cin nz, 16,
    // 2 cin nz ny bytes -- whose 8 x 32 x 6 x cin/8 x 1 box is one plane buffer.
    const auto enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(driver_tensor_map_encoder());
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap planes;
    const cuuint64_t dims[5] = {8, (cuuint64_t)nz, (cuuint64_t)ny, (cuuint64_t)(cin / 8), (cuuint64_t)nx};
    const cuuint64_t strides[4] = {(cuuint64_t)cin * 2, (cuuint64_t)nz * cin * 2, 16, (cuuint64_t)ny * nz * cin * 2};
    const cuuint32_t box[5] = {8, 32, 6, (cuuint32_t)(cin / 8), 1};
    const cuuint32_t elem[5] = {1, 1, 1, 1, 1};
    if (enc(&planes, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16 *>(in), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
#define TT_CONV_LAUNCH(CI, CO, R, F)                                                                  \
    do {                                                                                              \
        auto kern = k_conv3d_fwd_tc<CI, CO, R, F>;                                                    \
        /* at least 80 KB: no more than two CTAs share an SM's tensor memory */                     \
        constexpr uint32_t sm = TcConvSmem<CI, CO>::bytes > 80u * 1024u ? TcConvSmem<CI, CO>::bytes   \
                                                                        : 80u * 1024u;                 \
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);             \
        const long long slots = (long long)sm_count() * (sm <= 110u * 1024u ? 2 : 1);                  \
        const long long n_tiles = (long long)nx * tiles_y * tiles_z;                                   \
        const int grid = (int)(n_tiles < slots ? n_tiles : slots);                                     \
        kern<<<grid, kTcThreads, sm, st>>>(planes, wk, out, nx, ny, nz, tiles_y, tiles_z);            \
        return cudaGetLastError();                                                                    \
    } while (0)
    if (cin == 16 && cout == 32 && relu && !out_f32) TT_CONV_LAUNCH(16, 32, true, false);
    if (cin == 32 && cout == 32 && relu && !out_f32) TT_CONV_LAUNCH(32, 32, true, false);
    if (cin == 32 && cout == 16 && !relu && out_f32) TT_CONV_LAUNCH(32, 16, false, true);
    if (cin == 32 && cout == 32 && !relu && !out_f32) TT_CONV_LAUNCH(32, 32, false, false);
    if (cin == 16 && cout == 32 && !relu && !out_f32) TT_CONV_LAUNCH(16, 32, false, false);
    if (cin == 32 && cout == 16 && !relu && !out_f32) TT_CONV_LAUNCH(32, 16, false, false);
    if (cin == 16 && cout == 16 && !relu && out_f32) TT_CONV_LAUNCH(16, 16, false, true);
    if (cin == 16 && cout == 32 && !relu && out_f32) TT_CONV_LAUNCH(16, 32, false, true);
    if (cin == 32 && cout == 32 && !relu && out_f32) TT_CONV_LAUNCH(32, 32, false, true);
#undef TT_CONV_LAUNCH
    return cudaErrorInvalidValue;
}

cudaError_t conv3d_wgrad(const __nv_bfloat16 *x, const __nv_bfloat16 *dy, float *dw, int nx, int ny, int nz, int cin,
                         int cout, cudaStream_t st)
{
    const long long nseg = (long long)nx * ny * ((nz + 15) / 16);
    long long bx = (nseg + 63) / 64;
    if (bx > 24) bx = 24;
    if (bx < 1) bx = 1;
    const dim3 grid((unsigned)bx, 27);
    if (cin == 16 && cout == 32) k_conv3d_wgrad<16, 32><<<grid, 256, 0, st>>>(x, dy, dw, nx, ny, nz);
    else if (cin == 32 && cout == 32) k_conv3d_wgrad<32, 32><<<grid, 256, 0, st>>>(x, dy, dw, nx, ny, nz);
    else if (cin == 32 && cout == 16) k_conv3d_wgrad<32, 16><<<grid, 256, 0, st>>>(x, dy, dw, nx, ny, nz);
    else if (cin == 16 && cout == 16) k_conv3d_wgrad<16, 16><<<grid, 256, 0, st>>>(x, dy, dw, nx, ny, nz);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace tt

// ------------------------------------------------------- warm-start network

namespace tt {

__global__ void k_reduce(const double *__restrict__ partials, long long n, double *__restrict__ out,
                         const double *__restrict__ add, double mul);   // tt_misc.cu

constexpr int kNetLayers = 4;
constexpr int kHidden = 32;

static int layer_cin(int l) { return l == 0 ? 16 : kHidden; }
static int layer_cout(int l) { return l == kNetLayers - 1 ? 16 : kHidden; }
static int wsize(int l) { return 27 * layer_cout(l) * layer_cin(l); }

}  // namespace tt

using namespace tt;

struct tt_wsnet {
    int kin = 0, kout = 0;
    cudaStream_t stream = nullptr;
    int loss_blocks = 0;                 // CTAs of the loss reduction (four per SM)
    float *w[kNetLayers] = {}, *gw[kNetLayers] = {}, *m[kNetLayers] = {}, *v[kNetLayers] = {};
    __nv_bfloat16 *wk[kNetLayers] = {}, *wt[kNetLayers] = {};
    long long step = 0;
    long long cap = 0;                   // voxels the activation buffers hold
    __nv_bfloat16 *a[kNetLayers] = {};   // a[0] input (16 channels), a[1..3] hidden (32)
    float *out = nullptr;                // [nvox][16]
    __nv_bfloat16 *d0 = nullptr, *d1 = nullptr, *dout = nullptr;
    double *partials = nullptr, *loss_dev = nullptr, *loss_pinned = nullptr;
};

#define TT_NET_CUDA(call, what)                                    \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::tt::cuda_fail(_e, what);   \
    } while (0)

static void free_net_buffers(tt_wsnet *n)
{
    for (int l = 0; l < kNetLayers; ++l) { cudaFree(n->a[l]); n->a[l] = nullptr; }
    cudaFree(n->out); cudaFree(n->d0); cudaFree(n->d1); cudaFree(n->dout);
    n->out = nullptr; n->d0 = n->d1 = n->dout = nullptr;
    n->cap = 0;
}

static void free_net(tt_wsnet *n)
{
    if (!n) return;
    free_net_buffers(n);
    for (int l = 0; l < kNetLayers; ++l) {
        cudaFree(n->w[l]); cudaFree(n->gw[l]); cudaFree(n->m[l]); cudaFree(n->v[l]);
        cudaFree(n->wk[l]); cudaFree(n->wt[l]);
    }
    cudaFree(n->partials); cudaFree(n->loss_dev);
    if (n->loss_pinned) cudaFreeHost(n->loss_pinned);
    delete n;
}

static tt_status ensure_buffers(tt_wsnet *n, long long nvox)
{
    if (nvox <= n->cap) return TT_OK;
    free_net_buffers(n);
    TT_NET_CUDA(cudaMalloc(&n->a[0], sizeof(__nv_bfloat16) * nvox * 16), "wsnet buffers");
    for (int l = 1; l < kNetLayers; ++l)
        TT_NET_CUDA(cudaMalloc(&n->a[l], sizeof(__nv_bfloat16) * nvox * kHidden), "wsnet buffers");
    TT_NET_CUDA(cudaMalloc(&n->out, sizeof(float) * nvox * 16), "wsnet buffers");
    TT_NET_CUDA(cudaMalloc(&n->d0, sizeof(__nv_bfloat16) * nvox * kHidden), "wsnet buffers");
    TT_NET_CUDA(cudaMalloc(&n->d1, sizeof(__nv_bfloat16) * nvox * kHidden), "wsnet buffers");
    TT_NET_CUDA(cudaMalloc(&n->dout, sizeof(__nv_bfloat16) * nvox * 16), "wsnet buffers");
    n->cap = nvox;
    return TT_OK;
}

static tt_status cast_weights(tt_wsnet *n)
{
    for (int l = 0; l < kNetLayers; ++l) {
        const int co = layer_cout(l), ci = layer_cin(l);
        k_cast_conv_weights<<<grid_n(wsize(l)), 256, 0, n->stream>>>(n->w[l], co, ci, 0, n->wk[l]);
        k_cast_conv_weights<<<grid_n(wsize(l)), 256, 0, n->stream>>>(n->w[l], co, ci, 1, n->wt[l]);
    }
    TT_NET_CUDA(cudaGetLastError(), "wsnet weight cast");
    return TT_OK;
}

// net(x * in_scale) into n->out [nvox][16] (float).
static tt_status net_forward(tt_wsnet *n, int nx, int ny, int nz, const float *x, double in_scale)
{
    const long long nvox = (long long)nx * ny * nz;
    tt_status st = ensure_buffers(n, nvox);
    if (st != TT_OK) return st;
    k_pack_bf16<<<grid_n(nvox * 16), 256, 0, n->stream>>>(x, n->kin, nvox, (float)in_scale, n->a[0]);
    TT_NET_CUDA(cudaGetLastError(), "wsnet pack");
    for (int l = 0; l < kNetLayers; ++l) {
        const bool last = l == kNetLayers - 1;
        TT_NET_CUDA(conv3d_forward(n->a[l], n->wk[l], last ? (void *)n->out : (void *)n->a[l + 1], nx, ny, nz,
                                   layer_cin(l), layer_cout(l), !last, last, n->stream),
                    "wsnet conv forward");
    }
    return TT_OK;
}

// mean((net(x / in_scale) - target / out_scale)^2) and its weight gradients in n->gw.
static tt_status net_gradient(tt_wsnet *n, int nx, int ny, int nz, const float *x, const float *tgt, double in_scale,
                              double out_scale, double *loss_host)
{
    const long long nvox = (long long)nx * ny * nz;
    tt_status st = net_forward(n, nx, ny, nz, x, 1.0 / in_scale);
    if (st != TT_OK) return st;
    const double count = (double)nvox * n->kout;
    k_sq_error<<<n->loss_blocks, 256, 0, n->stream>>>(n->out, tgt, (float)(1.0 / out_scale), n->kout, nvox, 1.0 / count,
                                                     n->dout, n->partials);
    TT_NET_CUDA(cudaGetLastError(), "wsnet loss");
    k_reduce<<<1, 256, 0, n->stream>>>(n->partials, n->loss_blocks, n->loss_dev, nullptr, 1.0 / count);
    TT_NET_CUDA(cudaGetLastError(), "wsnet loss reduce");
    for (int l = 0; l < kNetLayers; ++l)
        TT_NET_CUDA(cudaMemsetAsync(n->gw[l], 0, sizeof(float) * wsize(l), n->stream), "wsnet memset");
    // backward; d = dL/d(pre-activation of layer l)
    __nv_bfloat16 *d = n->dout;
    for (int l = kNetLayers - 1; l >= 0; --l) {
        TT_NET_CUDA(conv3d_wgrad(n->a[l], d, n->gw[l], nx, ny, nz, layer_cin(l), layer_cout(l), n->stream),
                    "wsnet weight gradient");
        if (l == 0) break;
        __nv_bfloat16 *dn = (d == n->d0) ? n->d1 : n->d0;
        TT_NET_CUDA(conv3d_forward(d, n->wt[l], dn, nx, ny, nz, layer_cout(l), layer_cin(l), false, false, n->stream),
                    "wsnet data gradient");
        k_relu_mask<<<grid_n(nvox * kHidden), 256, 0, n->stream>>>(n->a[l], dn, nvox * kHidden);
        TT_NET_CUDA(cudaGetLastError(), "wsnet relu mask");
        d = dn;
    }
    TT_NET_CUDA(cudaMemcpyAsync(n->loss_pinned, n->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, n->stream),
                "wsnet loss copy");
    TT_NET_CUDA(cudaStreamSynchronize(n->stream), "stream synchronize");
    if (loss_host) *loss_host = *n->loss_pinned;
    return TT_OK;
}

static bool bad_dims(int nx, int ny, int nz) { return nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 28); }

extern "C" {

int tt_wsnet_num_weights(int k_in, int k_out)
{
    if (k_in < 1 || k_in > 16 || k_out < 1 || k_out > 16) return 0;
    return 27 * (kHidden * k_in + 2 * kHidden * kHidden + k_out * kHidden);
}

tt_status tt_wsnet_create(int k_in, int k_out, const float *w_host, void *stream, tt_wsnet **out)
{
    if (!out) { set_error("tt_wsnet_create: out must not be NULL"); return TT_INVALID_ARG; }
    *out = nullptr;
    if (k_in < 1 || k_in > 16 || k_out < 1 || k_out > 16 || !w_host) {
        set_error("tt_wsnet_create: need 1 <= k_in, k_out <= 16 and initial weights");
        return TT_INVALID_ARG;
    }
    tt_wsnet *n = new tt_wsnet();
    n->kin = k_in;
    n->kout = k_out;
    n->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < kNetLayers && e == cudaSuccess; ++l) {
        const size_t b = sizeof(float) * wsize(l);
        if (e == cudaSuccess) e = cudaMalloc(&n->w[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&n->gw[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&n->m[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&n->v[l], b);
        if (e == cudaSuccess) e = cudaMalloc(&n->wk[l], sizeof(__nv_bfloat16) * wsize(l));
        if (e == cudaSuccess) e = cudaMalloc(&n->wt[l], sizeof(__nv_bfloat16) * wsize(l));
        if (e == cudaSuccess) e = cudaMemsetAsync(n->m[l], 0, b, n->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(n->v[l], 0, b, n->stream);
    }
    n->loss_blocks = 4 * sm_count();
    if (e == cudaSuccess) e = cudaMalloc(&n->partials, sizeof(double) * n->loss_blocks);
    if (e == cudaSuccess) e = cudaMalloc(&n->loss_dev, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&n->loss_pinned, sizeof(double));
    if (e != cudaSuccess) { free_net(n); return cuda_fail(e, "tt_wsnet_create"); }
    // host weights [layer][27][co_real][ci_real] -> padded [27][COUT][CIN]
    const float *src = w_host;
    for (int l = 0; l < kNetLayers; ++l) {
        const int co = layer_cout(l), ci = layer_cin(l);
        const int cor = (l == kNetLayers - 1) ? k_out : kHidden, cir = (l == 0) ? k_in : kHidden;
        std::vector<float> pad((size_t)wsize(l), 0.f);
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < cor; ++o)
                for (int i = 0; i < cir; ++i) pad[((size_t)t * co + o) * ci + i] = src[((size_t)t * cor + o) * cir + i];
        src += (size_t)27 * cor * cir;
        e = cudaMemcpy(n->w[l], pad.data(), sizeof(float) * pad.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) { free_net(n); return cuda_fail(e, "tt_wsnet_create: weights"); }
    }
    tt_status st = cast_weights(n);
    if (st == TT_OK) {
        e = cudaStreamSynchronize(n->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "tt_wsnet_create");
    }
    if (st != TT_OK) { free_net(n); return st; }
    *out = n;
    return TT_OK;
}

tt_status tt_wsnet_destroy(tt_wsnet *n)
{
    free_net(n);
    return TT_OK;
}

tt_status tt_wsnet_set_stream(tt_wsnet *n, void *stream)
{
    if (!n) { set_error("null network"); return TT_INVALID_ARG; }
    n->stream = (cudaStream_t)stream;
    return TT_OK;
}

tt_status tt_wsnet_forward(tt_wsnet *n, int nx, int ny, int nz, const float *x, double in_scale, double out_scale,
                           float *y)
{
    if (!n || !x || !y || bad_dims(nx, ny, nz) || !(in_scale > 0) || !(out_scale > 0)) {
        set_error("tt_wsnet_forward: bad arguments");
        return TT_INVALID_ARG;
    }
    tt_status st = net_forward(n, nx, ny, nz, x, 1.0 / in_scale);
    if (st != TT_OK) return st;
    const long long nvox = (long long)nx * ny * nz;
    k_unpack_f32<<<grid_n(nvox * n->kout), 256, 0, n->stream>>>(n->out, n->kout, nvox, (float)out_scale, y);
    TT_NET_CUDA(cudaGetLastError(), "wsnet unpack");
    return TT_OK;
}

tt_status tt_wsnet_gradient(tt_wsnet *n, int nx, int ny, int nz, const float *x, const float *target,
                            double in_scale, double out_scale, float *grad_host, double *loss_host)
{
    if (!n || !x || !target || bad_dims(nx, ny, nz) || !(in_scale > 0) || !(out_scale > 0)) {
        set_error("tt_wsnet_gradient: bad arguments");
        return TT_INVALID_ARG;
    }
    tt_status st = net_gradient(n, nx, ny, nz, x, target, in_scale, out_scale, loss_host);
    if (st != TT_OK || !grad_host) return st;
    float *dst = grad_host;
    for (int l = 0; l < kNetLayers; ++l) {
        const int co = layer_cout(l), ci = layer_cin(l);
        const int cor = (l == kNetLayers - 1) ? n->kout : kHidden, cir = (l == 0) ? n->kin : kHidden;
        std::vector<float> pad((size_t)wsize(l));
        TT_NET_CUDA(cudaMemcpy(pad.data(), n->gw[l], sizeof(float) * pad.size(), cudaMemcpyDeviceToHost), "grad copy");
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < cor; ++o)
                for (int i = 0; i < cir; ++i) dst[((size_t)t * cor + o) * cir + i] = pad[((size_t)t * co + o) * ci + i];
        dst += (size_t)27 * cor * cir;
    }
    return TT_OK;
}

tt_status tt_wsnet_train_step(tt_wsnet *n, int nx, int ny, int nz, const float *x, const float *target,
                              double in_scale, double out_scale, double lr, double *loss_host)
{
    if (!n || !x || !target || bad_dims(nx, ny, nz) || !(in_scale > 0) || !(out_scale > 0) || !(lr > 0)) {
        set_error("tt_wsnet_train_step: bad arguments");
        return TT_INVALID_ARG;
    }
    tt_status st = net_gradient(n, nx, ny, nz, x, target, in_scale, out_scale, loss_host);
    if (st != TT_OK) return st;
    n->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
    for (int l = 0; l < kNetLayers; ++l)
        k_adam<<<grid_n(wsize(l)), 256, 0, n->stream>>>(n->w[l], n->gw[l], n->m[l], n->v[l], wsize(l), (float)lr, b1,
                                                         b2, 1e-8f, c1, c2);
    TT_NET_CUDA(cudaGetLastError(), "wsnet adam");
    return cast_weights(n);
}

tt_status tt_wsnet_get_weights(tt_wsnet *n, float *w_host)
{
    if (!n || !w_host) { set_error("tt_wsnet_get_weights: bad arguments"); return TT_INVALID_ARG; }
    TT_NET_CUDA(cudaStreamSynchronize(n->stream), "stream synchronize");
    float *dst = w_host;
    for (int l = 0; l < kNetLayers; ++l) {
        const int co = layer_cout(l), ci = layer_cin(l);
        const int cor = (l == kNetLayers - 1) ? n->kout : kHidden, cir = (l == 0) ? n->kin : kHidden;
        std::vector<float> pad((size_t)wsize(l));
        TT_NET_CUDA(cudaMemcpy(pad.data(), n->w[l], sizeof(float) * pad.size(), cudaMemcpyDeviceToHost), "weight copy");
        for (int t = 0; t < 27; ++t)
            for (int o = 0; o < cor; ++o)
                for (int i = 0; i < cir; ++i) dst[((size_t)t * cor + o) * cir + i] = pad[((size_t)t * co + o) * ci + i];
        dst += (size_t)27 * cor * cir;
    }
    return TT_OK;
}

// Single convolution for tests: y = conv(x, w) (+ ReLU), x [nvox][cin]
// bfloat16 (raw 16-bit), w [27][cout][cin] bfloat16, y [nvox][cout] float.
tt_status tt_conv3d_bf16(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, int relu, float *y,
                         void *stream)
{
    if (!x || !w || !y || bad_dims(nx, ny, nz) || (cin != 16 && cin != 32) || (cout != 16 && cout != 32)) {
        set_error("tt_conv3d_bf16: bad arguments");
        return TT_INVALID_ARG;
    }
    if (relu) { set_error("tt_conv3d_bf16: float output is compiled without ReLU"); return TT_UNSUPPORTED; }
    TT_NET_CUDA(conv3d_forward((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)w, y, nx, ny, nz, cin, cout, false,
                               true, (cudaStream_t)stream),
                "tt_conv3d_bf16");
    return TT_OK;
}

// The network's hidden-layer form: y = conv(x, w), ReLU optional, y
// [nvox][cout] bfloat16 (raw 16-bit), the output rounded once from the FP32
// accumulation.
tt_status tt_conv3d_bf16_act(int nx, int ny, int nz, int cin, int cout, const void *x, const void *w, int relu,
                             void *y, void *stream)
{
    if (!x || !w || !y || bad_dims(nx, ny, nz) || (cin != 16 && cin != 32) || (cout != 16 && cout != 32)) {
        set_error("tt_conv3d_bf16_act: bad arguments");
        return TT_INVALID_ARG;
    }
    if ((cin == 16 && cout == 16) || (relu && cout != 32)) {
        set_error("tt_conv3d_bf16_act: compiled for (cin, cout) = (16, 32), (32, 32) and, without ReLU, (32, 16)");
        return TT_UNSUPPORTED;
    }
    TT_NET_CUDA(conv3d_forward((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)w, y, nx, ny, nz, cin, cout,
                               relu != 0, false, (cudaStream_t)stream),
                "tt_conv3d_bf16_act");
    return TT_OK;
}

// Weight gradient for tests: dw [27][cout][cin] float += sum_v dy[v][co] x[v + d_t][ci].
tt_status tt_conv3d_wgrad_bf16(int nx, int ny, int nz, int cin, int cout, const void *x, const void *dy, float *dw,
                               void *stream)
{
    if (!x || !dy || !dw || bad_dims(nx, ny, nz) || (cin != 16 && cin != 32) || (cout != 16 && cout != 32)) {
        set_error("tt_conv3d_wgrad_bf16: bad arguments");
        return TT_INVALID_ARG;
    }
    TT_NET_CUDA(conv3d_wgrad((const __nv_bfloat16 *)x, (const __nv_bfloat16 *)dy, dw, nx, ny, nz, cin, cout,
                             (cudaStream_t)stream),
                "tt_conv3d_wgrad_bf16");
    return TT_OK;
}

}  // extern "C"
