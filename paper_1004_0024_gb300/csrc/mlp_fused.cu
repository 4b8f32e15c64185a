// The learned proposal's network (33 -> 256 -> 256 -> 32, ReLU) in one
// tcgen05 kernel: logits = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for tiles of
// 128 rows, bf16 operands, FP32 accumulation in tensor memory.
//
// Per block (one per SM, persistent over tiles), shared memory holds W1 and
// W3 for the whole launch, two X tiles, the 128 x 256 hidden activation H and
// two 32 KB buffers through which the four K chunks of W2 stream from L2 with
// 1-D bulk copies.  Thread 0 issues the bulk copies and the MMAs; the four
// warps run the epilogues (TMEM -> +bias, ReLU -> bf16 -> H in the operand
// layout), so H1 and H2 never leave the SM.  Accumulators: 256 TMEM columns,
// reused by the three layers.  Every wait is bounded; on timeout the error
// flag is raised, outstanding copies and MMAs are drained (bounded), TMEM is
// freed and the block returns.
#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace isg {
namespace {

constexpr long long kPolls = 1LL << 22;
constexpr int kXTile = 128 * 128;     // bytes of one X tile (128 rows x 64 bf16)
constexpr int kW1 = 256 * 128;        // W1 tile bytes
constexpr int kW3Chunk = 32 * 128;    // one K chunk of W3
constexpr int kW2Chunk = 256 * 128;   // one K chunk of W2
constexpr int kHChunk = 128 * 128;    // one K chunk of H
constexpr int kOffW1 = 0;
constexpr int kOffW3 = kOffW1 + kW1;
constexpr int kOffX = kOffW3 + 4 * kW3Chunk;
constexpr int kOffH = kOffX + 2 * kXTile;
constexpr int kOffW2 = kOffH + 4 * kHChunk;
constexpr int kSmem = kOffW2 + 2 * kW2Chunk;  // 212992 bytes

// Phase bookkeeping of one mbarrier as seen by the thread that waits on it.
struct Phase {
    uint32_t issued = 0, waited = 0;
};

__device__ __forceinline__ bool wait_next(uint64_t* bar, Phase& ph)
{
    if (!mbar_wait(bar, ph.waited & 1u, kPolls))
        return false;
    ++ph.waited;
    return true;
}

// bounded drain of every issued phase (used after a timeout)
__device__ __forceinline__ void drain(uint64_t* bar, Phase& ph)
{
    while (ph.waited < ph.issued)
        if (!wait_next(bar, ph))
            return;
}

// Epilogue of a 256-column accumulator: row 32 warp + lane, + bias, ReLU,
// bf16, written to H in the operand layout (4 K chunks of 128 rows).
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, int warp, int lane, const float* bias,
                                                unsigned char* H)
{
    const int row = 32 * warp + lane;
#pragma unroll 1
    for (int n0 = 0; n0 < 256; n0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(n0), v);
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float x0 = fmaxf(v[2 * i] + bias[n0 + 2 * i], 0.f);
            const float x1 = fmaxf(v[2 * i + 1] + bias[n0 + 2 * i + 1], 0.f);
            const __nv_bfloat162 p = __floats2bfloat162_rn(x0, x1);
            w[i] = *reinterpret_cast<const uint32_t*>(&p);
        }
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const int k = n0 + 8 * g;
            *reinterpret_cast<uint4*>(H + tiled_offset(128, row, k)) =
                make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
        }
    }
}

__global__ void __launch_bounds__(128, 1) mlp_fused_kernel(const MlpFusedArgs a)
{
    constexpr uint32_t IDESC256 = tc::idesc_bf16(128, 256);
    constexpr uint32_t IDESC32 = tc::idesc_bf16(128, 32);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t bar_w, bar_x[2], bar_full[2], bar_free[2], bar_mma;
    __shared__ float sb1[256], sb2[256], sb3[32];
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned char* gX = static_cast<const unsigned char*>(a.X);
    const unsigned char* gW2 = static_cast<const unsigned char*>(a.W2t);
    unsigned char* H = smem + kOffH;

    for (int i = tid; i < 256; i += 128) {
        sb1[i] = a.b1[i];
        sb2[i] = a.b2[i];
    }
    if (tid < 32)
        sb3[tid] = a.b3[tid];
    if (warp == 0)
        tc::tmem_alloc(&tslot, 256);
    if (tid == 0) {
        mbar_init(&bar_w, 1);
        mbar_init(&bar_mma, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_x[b], 1);
            mbar_init(&bar_full[b], 1);
            mbar_init(&bar_free[b], 1);
        }
        s_ok = 1;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;

    // phase counters, meaningful in thread 0 (the only thread that issues)
    Phase ph_w, ph_x[2], ph_full[2], ph_free[2], ph_mma;
    const int G = gridDim.x;
    const int n_it = int(blockIdx.x) < a.tiles ? (a.tiles - 1 - int(blockIdx.x)) / G + 1 : 0;
    auto load_x = [&](int it) {
        const int b = it & 1;
        const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
        mbar_expect_tx(&bar_x[b], kXTile);
        bulk_g2s(smem + kOffX + b * kXTile, gX + tile * kXTile, kXTile, &bar_x[b]);
        ++ph_x[b].issued;
    };
    auto load_w2 = [&](uint32_t n) {  // K chunk n & 3 of W2 into buffer n & 1
        const int b = int(n & 1u);
        mbar_expect_tx(&bar_full[b], kW2Chunk);
        bulk_g2s(smem + kOffW2 + b * kW2Chunk, gW2 + size_t(n & 3u) * kW2Chunk, kW2Chunk, &bar_full[b]);
        ++ph_full[b].issued;
    };
    if (tid == 0 && n_it > 0) {
        mbar_expect_tx(&bar_w, kW1 + 4 * kW3Chunk);
        bulk_g2s(smem + kOffW1, a.W1t, kW1, &bar_w);
        bulk_g2s(smem + kOffW3, a.W3t, 4 * kW3Chunk, &bar_w);
        ++ph_w.issued;
        load_x(0);
        if (n_it > 1)
            load_x(1);
        load_w2(0);
        load_w2(1);
    }

    // all threads observe each MMA completion (thread 0 first, bounded)
    uint32_t mma_seen = 0;
    auto observe = [&]() {
        if (tid != 0)
            mbar_wait(&bar_mma, mma_seen & 1u, kPolls);
        ++mma_seen;
        tc::fence_after_sync();
    };

    bool ok = true;
    for (int it = 0; it < n_it; ++it) {
        const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
        const int xb = it & 1;
        // ---- layer 1: D = X W1^T
        if (tid == 0) {
            bool good = (it > 0 || wait_next(&bar_w, ph_w)) && wait_next(&bar_x[xb], ph_x[xb]);
            if (good) {
                tc::fence_after_sync();
                const uint32_t xa = smem_u32(smem + kOffX + xb * kXTile), wa = smem_u32(smem + kOffW1);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem, tc::smem_desc(xa + kk * 256), tc::smem_desc(wa + kk * 256), IDESC256,
                                 kk > 0 ? 1u : 0u);
                tc::mma_commit(&bar_mma);
                ++ph_mma.issued;
                good = wait_next(&bar_mma, ph_mma);
                if (good && it + 2 < n_it)
                    load_x(it + 2);  // the buffer just read by layer 1
            }
            s_ok = good;
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        observe();
        hidden_epilogue(tmem, warp, lane, sb1, H);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // ---- layer 2: D = H1 W2^T, W2 streamed in four K chunks
        if (tid == 0) {
            tc::fence_after_sync();
            bool good = true;
            for (int c = 0; c < 4 && good; ++c) {
                const uint32_t n = 4u * uint32_t(it) + uint32_t(c);
                const int b = int(n & 1u);
                if (!(good = wait_next(&bar_full[b], ph_full[b])))
                    break;
                const uint32_t ha = smem_u32(H + c * kHChunk), wa = smem_u32(smem + kOffW2 + b * kW2Chunk);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem, tc::smem_desc(ha + kk * 256), tc::smem_desc(wa + kk * 256), IDESC256,
                                 (c > 0 || kk > 0) ? 1u : 0u);
                tc::mma_commit(&bar_free[b]);
                ++ph_free[b].issued;
                // refill the buffer of chunk n - 1 with chunk n + 1 once chunk n - 1's MMAs are done
                const bool next_exists = c < 3 || it + 1 < n_it;
                if (n >= 1u && next_exists) {
                    const int pb = int((n - 1u) & 1u);
                    if ((good = wait_next(&bar_free[pb], ph_free[pb])))
                        load_w2(n + 1u);
                }
            }
            if (good) {
                tc::mma_commit(&bar_mma);
                ++ph_mma.issued;
                good = wait_next(&bar_mma, ph_mma);
            }
            s_ok = good;
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        observe();
        hidden_epilogue(tmem, warp, lane, sb2, H);
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        // ---- layer 3: D[:, 0:32] = H2 W3^T
        if (tid == 0) {
            tc::fence_after_sync();
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const uint32_t ha = smem_u32(H + c * kHChunk), wa = smem_u32(smem + kOffW3 + c * kW3Chunk);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem, tc::smem_desc(ha + kk * 256), tc::smem_desc(wa + kk * 256), IDESC32,
                                 (c > 0 || kk > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar_mma);
            ++ph_mma.issued;
            s_ok = wait_next(&bar_mma, ph_mma);
        }
        __syncthreads();
        if (!s_ok) {
            ok = false;
            break;
        }
        observe();
        {
            float v[32];
            tc::tmem_ld32(tmem + (uint32_t(32 * warp) << 16), v);
            float* out = a.L + (tile * 128 + size_t(32 * warp + lane)) * 32;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                reinterpret_cast<float4*>(out)[i] = make_float4(v[4 * i] + sb3[4 * i], v[4 * i + 1] + sb3[4 * i + 1],
                                                                v[4 * i + 2] + sb3[4 * i + 2],
                                                                v[4 * i + 3] + sb3[4 * i + 3]);
        }
        tc::fence_before_sync();
        __syncthreads();  // TMEM reads done before the next tile's MMAs
    }
    if (!ok && tid == 0) {
        set_err(a.err, kErrTimeout);
        drain(&bar_mma, ph_mma);
        for (int b = 0; b < 2; ++b) {
            drain(&bar_free[b], ph_free[b]);
            drain(&bar_full[b], ph_full[b]);
            drain(&bar_x[b], ph_x[b]);
        }
        drain(&bar_w, ph_w);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(tmem, 256);
}

}  // namespace

cudaError_t mlp_fused_setup()
{
    return cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

cudaError_t launch_mlp_fused(const MlpFusedArgs& a, int grid, cudaStream_t st)
{
    if (a.tiles <= 0)
        return cudaSuccess;
    if (grid < 1)
        grid = 1;
    if (grid > a.tiles)
        grid = a.tiles;
    mlp_fused_kernel<<<grid, 128, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace isg
