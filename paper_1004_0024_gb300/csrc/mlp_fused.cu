// The learned proposal's network (33 -> 256 -> 256 -> 32, ReLU) in one
// tcgen05 kernel: logits = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for tiles of
// 128 rows, bf16 operands, FP32 accumulation in tensor memory.
//
// One CTA per SM, persistent over tiles, seventeen warps.  Warp 16 is the
// producer: it issues the 1-D bulk copies (W1, W2 and W3 once: all three stay
// resident in shared memory; X tiles double-buffered) and the MMAs.  Warps
// 0-15 run the epilogues.  Epilogue warp e reads the TMEM lanes of quadrant
// e % 4 (rows 32 (e % 4) .. +31) and the part k = e / 4 (64 columns) of the
// accumulator, 32 columns at a time: + bias, ReLU, bf16 pairs, stored back
// into TMEM in columns of its own part (the hidden activation is packed two
// per 32-bit column).  The next layer takes that activation as
// its A operand straight from TMEM, so H1 and H2 never leave tensor memory.
// Each 32-column step of all epilogue warps is signalled on its own mbarrier
// and the next layer's MMAs on that K range start while the warps convert
// the next step.
//
// TMEM (512 columns): layer 1 accumulates in 0..255 and H1 is packed in
// place into the first 32 columns of each 64-column part (columns the part's
// warp has read); layer 2 accumulates in 256..511 and H2 is packed in the
// same way; layer 3 accumulates in 288..319, the second half of part 0 of
// layer 2, once the epilogue of layer 2 is complete.  Layer 1 of the next
// tile (columns 0..255) is issued right after layer 2 of this one, so it runs
// while the warps convert layer 2; layer 2 of the next tile waits for the
// first step of its own epilogue, which follows the reads of layer 3.
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
constexpr int kW3Chunk = 32 * 128;    // one K chunk (64) of W3
constexpr int kW2Chunk = 256 * 128;   // one K chunk (64) of W2
constexpr int kOffW1 = 0;
constexpr int kOffW3 = kOffW1 + kW1;
constexpr int kOffW2 = kOffW3 + 4 * kW3Chunk;
constexpr int kOffX = kOffW2 + 4 * kW2Chunk;
constexpr int kSmem = kOffX + 2 * kXTile;  // 212992 bytes
constexpr int kEpiWarps = 16;              // four per TMEM lane quadrant
constexpr int kThreads = 32 * (kEpiWarps + 1);  // + 1 producer warp
constexpr int kParts = kEpiWarps / 4;      // column parts of a 256-column accumulator
constexpr int kPartCols = 256 / kParts;    // columns of one part (64)
constexpr int kSteps = kPartCols / 32;     // 32-column epilogue steps per part (2)
// TMEM column bases: H1 and H2 packed in place at the start of each part of
// D1 and D2; D3 in the second half of part 0 of D2 (read by its last step)
constexpr uint32_t kD1 = 0, kH1 = 0, kD2 = 256, kH2 = 256, kD3 = 256 + kPartCols / 2;

struct Bars {
    uint64_t w, x[2], m1, m2, m3, h1[kSteps], h2[kSteps];
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
    uint32_t issued = 0;
};

// relu(v + b) of two FP32 values as a bf16 pair (v0 + b0 in the low half):
// one packed FP32x2 add, then one converting instruction that also clamps
// negatives to zero
__device__ __forceinline__ uint32_t bias_relu_bf16x2(uint32_t v0, uint32_t v1, float b0, float b1)
{
    uint32_t r;
    asm("{ .reg .b64 v, b, s; .reg .f32 lo, hi;\n"
        "  mov.b64 v, {%1, %2};\n"
        "  mov.b64 b, {%3, %4};\n"
        "  add.rn.f32x2 s, v, b;\n"
        "  mov.b64 {lo, hi}, s;\n"
        "  cvt.rn.relu.bf16x2.f32 %0, hi, lo; }"
        : "=r"(r)
        : "r"(v0), "r"(v1), "f"(b0), "f"(b1));
    return r;
}

// Epilogue of a hidden layer by epilogue warp e, in kSteps steps j: the
// accumulator's columns dcol + kPartCols k + 32 j .. +31 (part k = e / 4) of
// the rows of lane quadrant e % 4: + bias, ReLU, bf16 pairs written to
// columns ocol + kPartCols k + 16 j .. +15 (K elements kPartCols k + 32 j ..
// +31 of the next layer), then an arrival on hbar[j].  With ocol = dcol the
// output goes into columns this warp has already read.  The load of step
// j + 1 is in flight while step j is converted and stored.
__device__ __forceinline__ void hidden_layer(uint32_t tmem, uint32_t dcol, uint32_t ocol, int e,
                                             const float* bias, uint64_t* hbar)
{
    const uint32_t lanes = uint32_t(32 * (e & 3)) << 16;
    const int k = e >> 2;
    uint32_t ra[32], rb[32];
    tc::tmem_ld32_async(tmem + lanes + dcol + uint32_t(kPartCols * k), ra);
    auto step = [&](int j, uint32_t (&cur)[32], uint32_t (&nxt)[32]) {
        tc::tmem_wait_ld(cur);
        if (j + 1 < kSteps)
            tc::tmem_ld32_async(tmem + lanes + dcol + uint32_t(kPartCols * k + 32 * (j + 1)), nxt);
        const int n0 = kPartCols * k + 32 * j;
        uint32_t w[16];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const float4 b = *reinterpret_cast<const float4*>(bias + n0 + 4 * i);
            w[2 * i] = bias_relu_bf16x2(cur[4 * i], cur[4 * i + 1], b.x, b.y);
            w[2 * i + 1] = bias_relu_bf16x2(cur[4 * i + 2], cur[4 * i + 3], b.z, b.w);
        }
        tc::tmem_st16(tmem + lanes + ocol + uint32_t(kPartCols * k + 16 * j), w);
        tc::tmem_wait_st();
        // the step's TMEM reads and writes are done before the arrival
        tc::fence_before_sync();
        mbar_arrive(&hbar[j]);
    };
#pragma unroll
    for (int j = 0; j < kSteps; ++j) {
        if (j & 1)
            step(j, rb, ra);
        else
            step(j, ra, rb);
    }
}

// Byte address of K elements k0 .. k0+15 of a weight matrix stored as K
// chunks of 64 (chunk bytes apart), each in the canonical layout
__device__ __forceinline__ uint32_t weight_k(uint32_t base, int chunk_bytes, int k0)
{
    return base + uint32_t((k0 >> 6) * chunk_bytes + ((k0 & 63) >> 4) * 256);
}

__global__ void __launch_bounds__(kThreads, 1) mlp_fused_kernel(const MlpFusedArgs a)
{
    constexpr uint32_t IDESC256 = tc::idesc_bf16(128, 256);
    constexpr uint32_t IDESC32 = tc::idesc_bf16(128, 32);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ Bars bars;
    __shared__ __align__(16) float sb1[256], sb2[256], sb3[32];
    __shared__ uint32_t tslot;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
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
        for (int b = 0; b < 2; ++b)
            mbar_init(&bars.x[b], 1);
        for (int c = 0; c < kSteps; ++c) {
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
            const uint32_t w1 = smem_u32(smem + kOffW1), w2 = smem_u32(smem + kOffW2),
                           w3 = smem_u32(smem + kOffW3);
            Phase ph_w, ph_x[2], ph_m1, ph_m2, ph_m3;
            auto load_x = [&](int it) {
                const int b = it & 1;
                const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
                mbar_expect_tx(&bars.x[b], kXTile);
                bulk_g2s(smem + kOffX + b * kXTile, gX + tile * kXTile, kXTile, &bars.x[b]);
                ++ph_x[b].issued;
            };
            auto commit = [&](uint64_t* bar, Phase& ph) {
                tc::mma_commit(bar);
                ++ph.issued;
            };
            auto mma1 = [&](int it) {  // D1 = X W1^T
                const uint32_t xa = smem_u32(smem + kOffX + (it & 1) * kXTile);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem + kD1, tc::smem_desc(xa + kk * 256), tc::smem_desc(w1 + kk * 256), IDESC256,
                                 kk > 0 ? 1u : 0u);
                commit(&bars.m1, ph_m1);
            };
            // the next layer on the K elements of epilogue step c:
            // kPartCols k + 32 c .. +31 of every part k, A packed in TMEM at
            // hcol + kPartCols k + 16 c
            auto mma_step = [&](uint32_t dcol, uint32_t hcol, uint32_t wbase, int chunk_bytes, uint32_t idesc,
                                int c) {
#pragma unroll
                for (int k = 0; k < kParts; ++k)
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int k0 = kPartCols * k + 32 * c + 16 * s;
                        tc::mma_bf16_tmem_a(tmem + dcol, tmem + hcol + uint32_t(kPartCols * k + 16 * c + 8 * s),
                                            tc::smem_desc(weight_k(wbase, chunk_bytes, k0)), idesc,
                                            (c == 0 && k == 0 && s == 0) ? 0u : 1u);
                    }
            };
            mbar_expect_tx(&bars.w, kW1 + 4 * kW3Chunk + 4 * kW2Chunk);
            bulk_g2s(smem + kOffW1, a.W1t, kW1, &bars.w);
            bulk_g2s(smem + kOffW3, a.W3t, 4 * kW3Chunk, &bars.w);
            for (int c = 0; c < 4; ++c)
                bulk_g2s(smem + kOffW2 + c * kW2Chunk, gW2 + size_t(c) * kW2Chunk, kW2Chunk, &bars.w);
            ++ph_w.issued;
            load_x(0);
            if (n_it > 1)
                load_x(1);
            bool ok = wait_phase(&bars.w, 0, abort) && wait_phase(&bars.x[0], 0, abort);
            if (ok) {
                tc::fence_after_sync();
                mma1(0);
            }
            for (int it = 0; ok && it < n_it; ++it) {
                const uint32_t par = uint32_t(it) & 1u;
                // X buffer of this tile is free once layer 1 has read it
                if (!(ok = wait_phase(&bars.m1, par, abort)))
                    break;
                if (it + 2 < n_it)
                    load_x(it + 2);
                // layer 2, step by step as the epilogue of layer 1 delivers H1
                for (int c = 0; c < kSteps && ok; ++c) {
                    if (!(ok = wait_phase(&bars.h1[c], par, abort)))
                        break;
                    tc::fence_after_sync();
                    mma_step(kD2, kH1, w2, kW2Chunk, IDESC256, c);
                }
                if (!ok)
                    break;
                commit(&bars.m2, ph_m2);
                // layer 1 of the next tile: columns 0..255 hold only this
                // tile's H1, read by the layer-2 MMAs issued before
                if (it + 1 < n_it) {
                    const int nb = (it + 1) & 1;
                    if (!(ok = wait_phase(&bars.x[nb], uint32_t((it + 1) >> 1) & 1u, abort)))
                        break;
                    tc::fence_after_sync();
                    mma1(it + 1);
                }
                // layer 3 once the epilogue of layer 2 has packed all of H2
                // (its last step has read the columns of D3)
                for (int c = 0; c < kSteps && ok; ++c)
                    ok = wait_phase(&bars.h2[c], par, abort);
                if (!ok)
                    break;
                tc::fence_after_sync();
                for (int c = 0; c < kSteps; ++c)
                    mma_step(kD3, kH2, w3, kW3Chunk, IDESC32, c);
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
                for (int b = 0; b < 2; ++b)
                    last(&bars.x[b], ph_x[b]);
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
            hidden_layer(tmem, kD1, kH1, warp, sb1, bars.h1);
            if (!wait_phase(&bars.m2, par, abort)) {
                fail();
                break;
            }
            tc::fence_after_sync();
            hidden_layer(tmem, kD2, kH2, warp, sb2, bars.h2);
            if (!wait_phase(&bars.m3, par, abort)) {
                fail();
                break;
            }
            tc::fence_after_sync();
            {  // the logits: warp e takes columns 8 (e / 4) .. +7 of its quadrant's
               // rows; the tile is stored column by column, so each store of
               // the warp writes 32 consecutive rows (128 bytes)
                const int quad = warp & 3, n0 = 8 * (warp >> 2);
                float v[8];
                tc::tmem_ld8(tmem + (uint32_t(32 * quad) << 16) + kD3 + uint32_t(n0), v);
                const size_t tile = size_t(blockIdx.x) + size_t(it) * G;
                float* out = a.L + tile * (128 * 32) + size_t(n0) * 128 + size_t(32 * quad + lane);
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    out[size_t(i) * 128] = v[i] + sb3[n0 + i];
            }
            // the D3 reads are done before the next tile's first arrival,
            // which layer 2 of that tile (overwriting D3) waits for
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
