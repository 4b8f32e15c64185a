// The learned proposal's network (33 -> 256 -> 256 -> 32, ReLU) in one
// tcgen05 kernel: logits = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for tiles of
// 128 rows, bf16 operands, FP32 accumulation in tensor memory.
//
// One CTA per SM, persistent over tiles, nine warps.  Warp 8 is the producer:
// it issues the 1-D bulk copies (W1 and W3 once, X tiles double-buffered, the
// four 32 KB K chunks of W2 streamed from L2 through two buffers) and the
// MMAs.  Warps 0-7 run the epilogues (warp e reads TMEM lanes = rows
// 32 (e % 4) .. +31 and half of each 64-column chunk): TMEM -> +bias, ReLU
// -> bf16 -> the hidden activation H in shared memory in the operand layout,
// 64 columns (one K chunk of the next
// layer) at a time, each chunk signalled on its own mbarrier so that the next
// layer's MMAs on that chunk start while the warps convert the next chunk.
// TMEM (512 columns): layer 1 accumulates in columns 0..255, layer 2 in
// 256..511 and layer 3 in 256..287 (free once layer 2's first chunk has been
// read), so layer 1 of the next tile overlaps layers 2 and 3 of this one.
// H1 and H2 never leave the SM.
//
// Every wait is bounded.  A role whose wait gives up raises the error flag
// and an abort flag the other roles poll; the producer then drains its
// outstanding copies and MMAs (bounded) and TMEM is freed before the CTA
// returns.
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
constexpr int kEpiWarps = 8;                  // two per TMEM lane quadrant
constexpr int kThreads = 32 * (kEpiWarps + 1);  // + 1 producer warp
constexpr uint32_t kD1 = 0, kD2 = 256, kD3 = 256;  // TMEM column bases

struct Bars {
    uint64_t w, x[2], full[2], free[2], m1, m2, m3, h1[4], h2[4];
};

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort)
{
    for (long long i = 0; i < kPolls; ++i) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if ((i & 1023) == 1023 && *abort)
            return false;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Phase bookkeeping of one mbarrier as seen by the producer.
struct Phase {
    uint32_t issued = 0, waited = 0;
};

// Epilogue of one 64-column chunk of a hidden layer by epilogue warp e: rows
// 32 (e % 4) + lane (the TMEM lanes of its quadrant), columns 32 (e / 4) ..
// +31 of the chunk: + bias, ReLU, bf16, written into K chunk c of H in the
// operand layout.
__device__ __forceinline__ void hidden_chunk(uint32_t tmem, uint32_t dcol, int c, int e, int lane,
                                             const float* bias, unsigned char* H)
{
    const int quad = e & 3, row = 32 * quad + lane;
    {
        const int n0 = 64 * c + 32 * (e >> 2);
        float v[32];
        tc::tmem_ld32(tmem + (uint32_t(32 * quad) << 16) + dcol + uint32_t(n0), v);
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
    // the chunk is visible to the tensor core and its TMEM reads are done
    tc::fence_proxy_async();
    tc::fence_before_sync();
}

__global__ void __launch_bounds__(kThreads, 1) mlp_fused_kernel(const MlpFusedArgs a)
{
    constexpr uint32_t IDESC256 = tc::idesc_bf16(128, 256);
    constexpr uint32_t IDESC32 = tc::idesc_bf16(128, 32);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Bars bars;
    __shared__ float sb1[256], sb2[256], sb3[32];
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* H = smem + kOffH;
    volatile int* abort = &s_abort;

    for (int i = tid; i < 256; i += kThreads) {
        sb1[i] = a.b1[i];
        sb2[i] = a.b2[i];
    }
    if (tid < 32)
        sb3[tid] = a.b3[tid];
    if (warp == 0)
        tc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        mbar_init(&bars.w, 1);
        mbar_init(&bars.m1, 1);
        mbar_init(&bars.m2, 1);
        mbar_init(&bars.m3, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bars.x[b], 1);
            mbar_init(&bars.full[b], 1);
            mbar_init(&bars.free[b], 1);
        }
        for (int c = 0; c < 4; ++c) {
            mbar_init(&bars.h1[c], 32 * kEpiWarps);
            mbar_init(&bars.h2[c], 32 * kEpiWarps);
        }
        s_abort = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;
    const int G = gridDim.x;
    const int n_it = int(blockIdx.x) < a.tiles ? (a.tiles - 1 - int(blockIdx.x)) / G + 1 : 0;
    auto fail = [&]() {
        set_err(a.err, kErrTimeout);
        *abort = 1;
    };

    if (warp == kEpiWarps) {
        // ------------------------------------------------------- producer
        if (lane == 0 && n_it > 0) {
            const unsigned char* gX = static_cast<const unsigned char*>(a.X);
            const unsigned char* gW2 = static_cast<const unsigned char*>(a.W2t);
            Phase ph_w, ph_x[2], ph_full[2], ph_free[2], ph_m1, ph_m2, ph_m3;
            auto load_x = [&](int it) {
                const int b = it & 1;
                const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
                mbar_expect_tx(&bars.x[b], kXTile);
                bulk_g2s(smem + kOffX + b * kXTile, gX + tile * kXTile, kXTile, &bars.x[b]);
                ++ph_x[b].issued;
            };
            auto load_w2 = [&](uint32_t n) {  // K chunk n & 3 of W2 into buffer n & 1
                const int b = int(n & 1u);
                mbar_expect_tx(&bars.full[b], kW2Chunk);
                bulk_g2s(smem + kOffW2 + b * kW2Chunk, gW2 + size_t(n & 3u) * kW2Chunk, kW2Chunk,
                         &bars.full[b]);
                ++ph_full[b].issued;
            };
            auto commit = [&](uint64_t* bar, Phase& ph) {
                tc::mma_commit(bar);
                ++ph.issued;
            };
            auto mma1 = [&](int it) {  // D1 = X W1^T
                const uint32_t xa = smem_u32(smem + kOffX + (it & 1) * kXTile), wa = smem_u32(smem + kOffW1);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem + kD1, tc::smem_desc(xa + kk * 256), tc::smem_desc(wa + kk * 256),
                                 IDESC256, kk > 0 ? 1u : 0u);
                commit(&bars.m1, ph_m1);
            };
            mbar_expect_tx(&bars.w, kW1 + 4 * kW3Chunk);
            bulk_g2s(smem + kOffW1, a.W1t, kW1, &bars.w);
            bulk_g2s(smem + kOffW3, a.W3t, 4 * kW3Chunk, &bars.w);
            ++ph_w.issued;
            load_x(0);
            if (n_it > 1)
                load_x(1);
            load_w2(0);
            load_w2(1);
            bool ok = wait_phase(&bars.w, 0, abort) && wait_phase(&bars.x[0], 0, abort);
            if (ok) {
                tc::fence_after_sync();
                mma1(0);
            }
            for (int it = 0; ok && it < n_it; ++it) {
                // X buffer of this tile is free once layer 1 has read it
                if (!(ok = wait_phase(&bars.m1, uint32_t(it) & 1u, abort)))
                    break;
                if (it + 2 < n_it)
                    load_x(it + 2);
                // layer 2, chunk by chunk as the epilogue of layer 1 delivers H1
                for (int c = 0; c < 4 && ok; ++c) {
                    const uint32_t n = 4u * uint32_t(it) + uint32_t(c);
                    const int b = int(n & 1u);
                    if (!(ok = wait_phase(&bars.full[b], (n >> 1) & 1u, abort) &&
                               wait_phase(&bars.h1[c], uint32_t(it) & 1u, abort)))
                        break;
                    tc::fence_after_sync();
                    const uint32_t ha = smem_u32(H + c * kHChunk), wa = smem_u32(smem + kOffW2 + b * kW2Chunk);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem + kD2, tc::smem_desc(ha + kk * 256), tc::smem_desc(wa + kk * 256),
                                     IDESC256, (c > 0 || kk > 0) ? 1u : 0u);
                    commit(&bars.free[b], ph_free[b]);
                    // refill the buffer of chunk n - 1 with chunk n + 1 once its MMAs are done
                    const bool next_exists = c < 3 || it + 1 < n_it;
                    if (n >= 1u && next_exists) {
                        const int pb = int((n - 1u) & 1u);
                        if ((ok = wait_phase(&bars.free[pb], ph_free[pb].waited & 1u, abort))) {
                            ++ph_free[pb].waited;
                            load_w2(n + 1u);
                        }
                    }
                }
                if (!ok)
                    break;
                commit(&bars.m2, ph_m2);
                // layer 1 of the next tile: D1 was last read by this tile's epilogue 1
                if (it + 1 < n_it) {
                    const int nb = (it + 1) & 1;
                    if (!(ok = wait_phase(&bars.x[nb], uint32_t((it + 1) >> 1) & 1u, abort)))
                        break;
                    tc::fence_after_sync();
                    mma1(it + 1);
                }
                // layer 3, chunk by chunk as the epilogue of layer 2 delivers H2
                for (int c = 0; c < 4 && ok; ++c) {
                    if (!(ok = wait_phase(&bars.h2[c], uint32_t(it) & 1u, abort)))
                        break;
                    tc::fence_after_sync();
                    const uint32_t ha = smem_u32(H + c * kHChunk), wa = smem_u32(smem + kOffW3 + c * kW3Chunk);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem + kD3, tc::smem_desc(ha + kk * 256), tc::smem_desc(wa + kk * 256),
                                     IDESC32, (c > 0 || kk > 0) ? 1u : 0u);
                }
                if (ok)
                    commit(&bars.m3, ph_m3);
            }
            if (!ok) {
                fail();
                // every barrier has at most one phase of its own copies / MMAs outstanding
                auto last = [&](uint64_t* bar, const Phase& ph) {
                    if (ph.issued > 0)
                        mbar_wait(bar, (ph.issued - 1u) & 1u, kPolls);
                };
                last(&bars.m1, ph_m1);
                last(&bars.m2, ph_m2);
                last(&bars.m3, ph_m3);
                for (int b = 0; b < 2; ++b) {
                    last(&bars.free[b], ph_free[b]);
                    last(&bars.full[b], ph_full[b]);
                    last(&bars.x[b], ph_x[b]);
                }
                last(&bars.w, ph_w);
            }
        }
    } else {
        // --------------------------------------------------- epilogue warps
        for (int it = 0; it < n_it; ++it) {
            const uint32_t par = uint32_t(it) & 1u;
            if (!wait_phase(&bars.m1, par, abort)) {
                fail();
                break;
            }
            tc::fence_after_sync();
            for (int c = 0; c < 4; ++c) {
                hidden_chunk(tmem, kD1, c, warp, lane, sb1, H);
                mbar_arrive(&bars.h1[c]);
            }
            if (!wait_phase(&bars.m2, par, abort)) {
                fail();
                break;
            }
            tc::fence_after_sync();
            for (int c = 0; c < 4; ++c) {
                hidden_chunk(tmem, kD2, c, warp, lane, sb2, H);
                mbar_arrive(&bars.h2[c]);
            }
            if (!wait_phase(&bars.m3, par, abort)) {
                fail();
                break;
            }
            tc::fence_after_sync();
            if (warp < 4) {  // the logits: one quadrant of rows per warp
                float v[32];
                tc::tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + kD3, v);
                const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
                float* out = a.L + (tile * 128 + size_t(32 * warp + lane)) * 32;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    reinterpret_cast<float4*>(out)[i] =
                        make_float4(v[4 * i] + sb3[4 * i], v[4 * i + 1] + sb3[4 * i + 1],
                                    v[4 * i + 2] + sb3[4 * i + 2], v[4 * i + 3] + sb3[4 * i + 3]);
            }
            tc::fence_before_sync();
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0)
        tc::tmem_dealloc(tmem, 512);
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
    mlp_fused_kernel<<<grid, kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace isg
