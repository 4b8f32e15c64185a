// bf16 GEMM on the 5th-generation tensor cores: C = epi(A B^T), FP32 in TMEM.
//
//   A [M][lda] and B [N][ldb] are bf16, row-major with K contiguous; M is a
//   multiple of 128, N one of 32/64/128/256 (one N tile per block), K a
//   multiple of 64.  Block b computes rows 128b .. 128b+127.
//   epi: + bias[n] (optional), ReLU (optional), zero where mask[m][n] <= 0
//   (optional, the ReLU derivative in back-propagation), then FP32 or bf16.
//
// Pipeline: four warps stage K chunks of 64 (A 16 KB, B N x 128 B) into shared
// memory with cp.async, two buffers deep; thread 0 issues four 128 x N x 16
// MMAs per chunk into one TMEM accumulator and commits them to the buffer's
// mbarrier; a buffer is refilled only after the MMAs that read it completed.
// The epilogue reads the accumulator with tcgen05.ld (warp w owns TMEM lanes
// = rows 32w .. 32w+31).  Every wait is bounded: on timeout the error flag is
// raised, the block waits (bounded) for its MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace isg {
namespace {

constexpr long long kPolls = 1LL << 22;

__device__ __forceinline__ void cp16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

template <int N>
__global__ void __launch_bounds__(128, 1) tc_gemm_kernel(const TcGemmArgs g)
{
    constexpr int NCOLS = N < 32 ? 32 : N;
    constexpr uint32_t IDESC = tc::idesc_bf16(128, N);
    constexpr int A_BYTES = 128 * 128;  // 128 rows x 64 bf16
    constexpr int B_BYTES = N * 128;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tslot;
    __shared__ int s_ok;
    unsigned char* sA[2] = {smem, smem + A_BYTES};
    unsigned char* sB[2] = {smem + 2 * A_BYTES, smem + 2 * A_BYTES + B_BYTES};
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128;
    const int nk = g.K / tc::kChunkK;
    const __nv_bfloat16* A = static_cast<const __nv_bfloat16*>(g.A);
    const __nv_bfloat16* B = static_cast<const __nv_bfloat16*>(g.B);

    if (warp == 0)
        tc::tmem_alloc(&tslot, NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tslot;

    auto stage = [&](int c, int buf) {
        const int k0 = c * tc::kChunkK;
        for (int idx = tid; idx < 128 * 8; idx += 128) {
            const int row = idx >> 3, kg = idx & 7;
            cp16(sA[buf] + tc::tile_offset(row, kg), A + size_t(m0 + row) * g.lda + k0 + kg * 8);
        }
        for (int idx = tid; idx < N * 8; idx += 128) {
            const int row = idx >> 3, kg = idx & 7;
            cp16(sB[buf] + tc::tile_offset(row, kg), B + size_t(row) * g.ldb + k0 + kg * 8);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
        tc::fence_proxy_async();
        __syncthreads();
    };
    // bounded wait on the commit of chunk c, decided by thread 0 for the block
    auto wait_chunk = [&](int c) -> bool {
        if (tid == 0)
            s_ok = mbar_wait(&mbar[c & 1], uint32_t((c >> 1) & 1), kPolls) ? 1 : 0;
        __syncthreads();
        if (s_ok)
            mbar_wait(&mbar[c & 1], uint32_t((c >> 1) & 1), kPolls);  // acquire in every thread
        return s_ok != 0;
    };

    bool ok = true;
    int issued = -1;
    stage(0, 0);
    for (int c = 0; c < nk; ++c) {
        const int buf = c & 1;
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t a0 = smem_u32(sA[buf]), b0 = smem_u32(sB[buf]);
#pragma unroll
            for (int kk = 0; kk < tc::kChunkK / 16; ++kk)
                tc::mma_bf16(tmem, tc::smem_desc(a0 + kk * 2 * tc::kLBO),
                             tc::smem_desc(b0 + kk * 2 * tc::kLBO), IDESC, (c > 0 || kk > 0) ? 1u : 0u);
            tc::mma_commit(&mbar[buf]);
        }
        issued = c;
        if (c + 1 < nk) {
            if (c >= 1 && !(ok = wait_chunk(c - 1)))
                break;
            stage(c + 1, (c + 1) & 1);
        }
    }
    if (ok)
        ok = wait_chunk(issued);
    if (!ok) {
        if (tid == 0)
            set_err(g.err, kErrTimeout);
        if (issued >= 0 && tid == 0)
            mbar_wait(&mbar[issued & 1], uint32_t((issued >> 1) & 1), kPolls);
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0)
            tc::tmem_dealloc(tmem, NCOLS);
        return;
    }
    tc::fence_after_sync();

    // ---- epilogue: row m0 + 32 warp + lane, 32 columns at a time
    const int row = m0 + 32 * warp + lane;
    const __nv_bfloat16* mrow =
        g.mask ? static_cast<const __nv_bfloat16*>(g.mask) + size_t(row) * g.ldm : nullptr;
#pragma unroll 1
    for (int n0 = 0; n0 < N; n0 += 32) {
        float v[32];
        tc::tmem_ld32(tmem + (uint32_t(32 * warp) << 16) + uint32_t(n0), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            float x = v[i];
            if (g.bias)
                x += g.bias[n0 + i];
            if (g.relu)
                x = fmaxf(x, 0.f);
            if (mrow && !(__bfloat162float(mrow[n0 + i]) > 0.f))
                x = 0.f;
            v[i] = x;
        }
        if (g.c_bf16) {
            __nv_bfloat16* out = static_cast<__nv_bfloat16*>(g.C) + size_t(row) * g.ldc + n0;
            uint32_t w[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                w[i] = *reinterpret_cast<const uint32_t*>(&p);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
                reinterpret_cast<uint4*>(out)[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
        } else {
            float* out = static_cast<float*>(g.C) + size_t(row) * g.ldc + n0;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                reinterpret_cast<float4*>(out)[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0)
        tc::tmem_dealloc(tmem, NCOLS);
}

template <int N>
size_t tc_smem_bytes()
{
    return size_t(2 * 128 * 128 + 2 * N * 128);
}

template <int N>
cudaError_t launch_n(const TcGemmArgs& g, cudaStream_t st)
{
    tc_gemm_kernel<N><<<g.M / 128, 128, tc_smem_bytes<N>(), st>>>(g);
    return cudaGetLastError();
}

}  // namespace

cudaError_t tc_gemm_setup()
{
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(tc_smem_bytes<32>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(tc_smem_bytes<64>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(tc_smem_bytes<128>()));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_gemm_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(tc_smem_bytes<256>()));
    return e;
}

cudaError_t launch_tc_gemm(const TcGemmArgs& g, cudaStream_t st)
{
    if (g.M <= 0 || g.M % 128 || g.K <= 0 || g.K % tc::kChunkK || g.lda % 8 || g.ldb % 8 ||
        g.ldc % 8 || (g.mask && g.ldm % 8))
        return cudaErrorInvalidValue;
    switch (g.N) {
    case 32: return launch_n<32>(g, st);
    case 64: return launch_n<64>(g, st);
    case 128: return launch_n<128>(g, st);
    case 256: return launch_n<256>(g, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace isg
