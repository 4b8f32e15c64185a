// Internal declarations of the GB300 Ising library (not part of the C ABI).
//
// Data layout (HBM):
//   spins   int8  [R][n]       slot-major, spin index order (API layout)
//   fields  int16|int32 [R][n] total local field f_i = h_i + sum_j J_ij s_j
//   E       int32 [R]          energy of each slot
// Per-slice tables (sorted position p = rank of site q by (slice level, q)):
//   nbr_off int32 [S+1], nbr uint32 [E] packed (pos(q') << 16 | (uint16)J),
//   jtau int32 [S] Trotter coupling, lev0 int32 [S] slice wavefront level,
//   site int32 [S] (site at position p), pos int32 [S] (position of site q).
// Inside a sweep block (shared memory), per replica g of the block:
//   colbits uint32 [S][G][W]  bit t of column (p, g) = spin (q, t) is +1
//   fsp     FT     [S][M][G]  spatial field h_q + sum_{q'} J s_{q',t}
//                             (int16 kept biased by +32768 inside 32-bit words)
// The Trotter part of the field, Jtau_q (s_{q,t-1} + s_{q,t+1}), is read from
// the column bits, so only the spatial part needs atomic updates.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace isg {

constexpr int kMtRing = 1024;  // ring slots of an MT19937 stream (>= 624 + 227)
constexpr int kMtStep = 227;   // words of one stream computable in parallel

// Device error flag values (first error wins).
constexpr int kErrTimeout = 1;
constexpr int kErrBadConfig = 2;

struct SweepArgs {
    // slice structure
    int S, M, W, N, D0, D, Mp;
    int K;          // flip-threshold table length: k in [1, K) tabulated, k >= K -> 0
    int G, R;       // replicas per block, replicas in total
    int nsweeps;    // sweeps in this launch
    int tables_smem;     // 1: stage tables in shared memory via bulk copies
    int thr_smem;        // 1: thresholds staged in shared memory
    int nbr_count;       // entries of nbr
    const int* nbr_off;
    const uint32_t* nbr;
    const int* jtau;
    const int* lev0;
    const int* site;
    const int* pos;
    // state
    int8_t* spins;
    void* fields;
    int* E;
    const int* temp_of_slot;
    const uint32_t* thr;  // [R temps][K]
    // random numbers
    int rng;              // 0 MT19937 (words from wbuf), 1 Philox
    uint32_t seed, inst;
    unsigned long long* counters;  // [0] sweeps done, [1] passes done
    const uint32_t* wbuf;          // MT words: [sweep][R][S][Mp]
    long long wbuf_sweep_stride;   // = R*S*Mp
    unsigned int* done_blocks;     // block-completion counter for the counter update
    int* err;
    // parallel tempering fused into a persistent (cooperative) launch
    int swap_every;                // 0: no PT pass inside this launch
    int* slot_of_temp;             // [R]
    int* temp_of_slot_out;         // [R] written back by block 0
    unsigned long long* swap_acc;  // [R-1]
    const uint32_t* swthr;
    const long long* swoff;
    const int* swlen;
    const uint32_t* swbuf;         // MT swap words [pass][maxpairs]
    int maxpairs;
    int* E_pub;                    // [2][R] energies published for the PT pass
    unsigned int* gridbar;         // grid barrier arrivals (zeroed before the launch)
    int lg_G;                      // log2(G)
    int inst_blocks;               // blocks of this instance (batched launches)
    // track schedule (track kernel): columns track_col[track_off[k] ..
    // track_off[k+1]) in time order form track k
    const int* track_off;
    const int* track_col;
    int ntracks;
    // generic kernel: stage each column's random words in shared memory,
    // two 4-word blocks ahead of use (cp.async for MT19937 words, one Philox
    // call per block), when the staging area fits; the host enables it for
    // MT19937 only
    int stage_words;
    // lean kernel: at most one owned column of a thread is busy per level
    // (no level has more busy columns than the block has threads)
    int one_active;
    // split couplings (ising_set_trotter; lean kernel only): the fields are
    // spatial, E the spatial energy, C = -sum over Trotter pairs of s s', and
    // the flip table of temperature k has K = 3 (2 split_ks + 1) entries, entry
    // (k_s + split_ks) * 3 + k_tau / 2 + 1 for k_s = s f_space in
    // [-split_ks, split_ks] and k_tau = s (s_{t-1} + s_{t+1}) in {-2, 0, 2}
    int split;
    int split_ks;
    int* C;                // [R]
    int* C_pub;            // [2][R] Trotter sums published for the PT pass
    const double* dbeta;   // [R-1] beta_{k+1} - beta_k
    const double* dK;      // [R-1] K_{k+1} - K_k
    // packed kernel (packed_impl.cuh): the table buffer (column descriptors,
    // positions, slot offsets, slot columns; pk_bytes long), the number of
    // slots, and the global field width (16 or 32)
    const uint32_t* pk;
    uint32_t pk_bytes;
    int nslots;
    int field_bits;
    // packed kernel, MT19937: with gen > 0, gen extra warps of each block
    // advance the replica's stream (ring [R + 1][kMtRing], positions) and
    // write the next sweep's words into a two-sweep buffer (wbuf, parity of
    // the sweep) while the block's sweep_threads threads run the current one
    int gen;
    int gen_slices;  // MT19937: slices the generator stages per column store (4, or 2 to save shared memory; 0 = 4)
    uint32_t* mtring;
    unsigned long long* mtpos;
    int sweep_threads;
};

// One block of a batched launch: instance index and block index within it.
struct BatchItem {
    int inst, block;
};

struct PtArgs {
    int R;
    int* E;
    int* temp_of_slot;
    int* slot_of_temp;
    unsigned long long* swap_acc;
    unsigned long long* counters;
    const uint32_t* swthr;     // flattened swap thresholds
    const long long* swoff;    // [R-1] start of pair k's table
    const int* swlen;          // [R-1] table length (d in [1, len) tabulated)
    int rng;
    uint32_t seed, inst;
    const uint32_t* swbuf;     // MT swap words [pass][maxpairs]
    int maxpairs;
    int pass_rel;              // pass index inside swbuf
    // split couplings: z = dbeta dE + dK dC with the deterministic exponential
    int split;
    const int* C;              // [R]
    const double* dbeta;       // [R-1]
    const double* dK;          // [R-1]
};

struct MtGenArgs {
    uint32_t* ring;            // [streams][kMtRing]
    unsigned long long* pos;   // [streams] index w of the next x_w to generate
    int R;                     // replica streams 0..R-1, swap stream R
    int first_stream;          // block b generates stream first_stream + b
    int mode;                  // 0 sweep words, 1 initial spins
    long long nwords;          // words per replica stream
    int N, S, M, Mp;
    const int* pos_of_site;
    uint32_t* wbuf;
    long long wbuf_sweep_stride;
    int8_t* spins;
    // swap stream (block R when do_swap)
    int do_swap;
    int swap_passes;           // passes to cover
    uint32_t* swbuf;
    int maxpairs;
    const unsigned long long* counters;
};

// ------------------------------------------------------------------ RNG
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ uint32_t pick4(uint4 v, int lane)
{
    return (lane & 2) ? ((lane & 1) ? v.w : v.z) : ((lane & 1) ? v.y : v.x);
}

// MT19937 recurrence x_w = x_{w-227} ^ twist(x_{w-624}, x_{w-623}) and
// tempering (Matsumoto & Nishimura 1998).
__device__ __forceinline__ uint32_t mt_recur(uint32_t xa, uint32_t xb, uint32_t xm)
{
    const uint32_t y = (xa & 0x80000000u) | (xb & 0x7FFFFFFFu);
    return xm ^ (y >> 1) ^ ((0u - (y & 1u)) & 0x9908B0DFu);
}

__device__ __forceinline__ uint32_t mt_temper(uint32_t y)
{
    y ^= y >> 11;
    y ^= (y << 7) & 0x9D2C5680u;
    y ^= (y << 15) & 0xEFC60000u;
    y ^= y >> 18;
    return y;
}

// ------------------------------------------------ bulk copy (TMA) + mbarrier
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk global -> shared copy; dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bounded wait for phase `parity` of the barrier; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long max_polls)
{
    for (long long i = 0; i < max_polls; ++i) {
        uint32_t ok;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
    }
    return false;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned).
// Unlike a register load it is not waited for by bar.sync.
__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void set_err(int* err, int code)
{
    atomicCAS(err, 0, code);
}

// bf16 tensor-core GEMM C = epi(A B^T) (tc_gemm.cu).
struct TcGemmArgs {
    const void* A;      // bf16 [M][lda]
    const void* B;      // bf16 [N][ldb]
    int lda, ldb, M, N, K;
    const float* bias;  // [N] or null
    const void* mask;   // bf16 [M][ldm] or null: zero where mask <= 0
    int ldm, relu;
    void* C;            // [M][ldc], bf16 when c_bf16 else FP32
    int ldc, c_bf16;
    int* err;
};
cudaError_t tc_gemm_setup();
cudaError_t launch_tc_gemm(const TcGemmArgs& g, cudaStream_t st);

// The learned proposal's 3-layer network in one tcgen05 kernel (mlp_fused.cu).
// Operands are pre-tiled in the canonical K-major core-matrix layout of the
// shared-memory descriptors: X in tiles of 128 rows x 64 (16 KB each), W1
// [256][64] (32 KB), W2 [256][256] as four K chunks of 32 KB, W3 [32][256] as
// four K chunks of 4 KB.
struct MlpFusedArgs {
    const void* X;
    const void *W1t, *W2t, *W3t;
    const float *b1, *b2, *b3;  // [256], [256], [32]
    float* L;                   // [tiles][32][128] logits, each tile stored column by column
    int tiles;
    int* err;
};
cudaError_t mlp_fused_setup();
cudaError_t launch_mlp_fused(const MlpFusedArgs& a, int grid, cudaStream_t st);
// byte offset of element (row, k) of a K-major tile with `rows` rows in the
// core-matrix layout, K split into chunks of 64
__host__ __device__ __forceinline__ size_t tiled_offset(int rows, int row, int k)
{
    return size_t(k >> 6) * size_t(rows) * 128 + size_t(row >> 3) * 1024 + size_t((k & 63) >> 3) * 128 +
           size_t(row & 7) * 16 + size_t(k & 7) * 2;
}

// Largest block of the small-block lean instantiation (kernel variant 3: two
// columns per thread, eight resident blocks per SM).
constexpr int kLeanSmallThreads = 128;

// Everything needed to launch a handle's register-resident sweep kernel.
struct FusedLaunch {
    SweepArgs args;
    int field_bits, cmax, threads, blocks, R, rng;
    size_t smem_plain, smem_fused;
    int variant;  // 0 fast, 1 lean, 2 track, 3 lean with small blocks, 4 lean with long columns
    cudaStream_t stream;
};

// ---------------------------------------------------------- launchers
cudaError_t launch_sweep(const SweepArgs& a, int field_bits, int cmax, int threads, int blocks,
                         size_t smem, cudaStream_t st);
size_t sweep_smem_bytes(const SweepArgs& a, int field_bits);
cudaError_t sweep_set_smem_limits();
size_t sweep_max_dynamic_smem();
int sweep_cmax_for(int c);
cudaError_t sweep_max_blocks_per_sm(int field_bits, int cmax, int rng, int threads, size_t smem,
                                    int* out);
cudaError_t launch_pt(const PtArgs& a, cudaStream_t st);
// register-resident sweep for M <= 32 with tables in shared memory
// variant: 0 the register-resident kernel (fast_impl.cuh), 1 its lean
// one-replica form (lean_impl.cuh: G = 1, M in {4,8,16,32}, spatial degree
// <= 6, |J| <= 63, at most 4 columns per thread), 2 the track-scheduled form
// (track_impl.cuh: lean's limits, one thread per track, cmax unused)
size_t fast_smem_bytes(const SweepArgs& a, int field_bits, int variant = 0, int threads = 0);
cudaError_t fast_set_smem_limits();
// Batched launches: block b runs item items[b] with args[items[b].inst].
cudaError_t launch_fast_batch(const SweepArgs* args, const BatchItem* items, int n_items,
                              int field_bits, int rng, int cmax, int threads, size_t smem, int variant,
                              cudaStream_t st);
cudaError_t launch_pt_batch(const PtArgs* args, int n_inst, int max_R, cudaStream_t st);
// Packed kernel over ragged batches (one cooperative launch of whole
// instances, block b = items[b]; rmax: 1 or 2 slot rounds per thread).
cudaError_t fast_max_blocks_per_sm_batch(int rng, int rmax, int threads, size_t smem, int* out);
cudaError_t launch_packed_batch(const SweepArgs* args, const BatchItem* items, int n_items, int rng, int rmax,
                                int threads, size_t smem, cudaStream_t st);
cudaError_t launch_mt_gen_batch(const MtGenArgs* args, const BatchItem* items, int n_items,
                                int max_S, cudaStream_t st);
// split: the split-coupling instantiation of the lean kernel (variants 1, 3, 4
// only; launch_fast takes it from a.split)
cudaError_t fast_max_blocks_per_sm(int field_bits, int cmax, int rng, int threads, size_t smem,
                                   int* out, int variant = 0, bool split = false);
cudaError_t launch_fast(const SweepArgs& a, int field_bits, int cmax, int threads, int blocks,
                        size_t smem, bool cooperative, cudaStream_t st, int variant = 0);
cudaError_t launch_mt_gen(const MtGenArgs& a, int blocks, cudaStream_t st);
cudaError_t mt_gen_set_smem_limit();
cudaError_t launch_philox_init(int8_t* spins, int R, int N, int S, uint32_t seed, uint32_t inst,
                               cudaStream_t st);
cudaError_t launch_widen_i16(const int16_t* src, int* dst, long long n, cudaStream_t st);
cudaError_t launch_state_init(const int8_t* spins, void* fields, int field_bits, int* E, int R,
                              int N, const int* row_ptr, const int* col, const int* J,
                              const int* h, cudaStream_t st);
// Split couplings: spatial fields, spatial energy and Trotter sum C of every
// replica from its spins (an edge is spatial when both ends lie in one slice
// of S spins).
cudaError_t launch_split_state_init(const int8_t* spins, void* fields, int field_bits, int* E, int* C,
                                    int R, int N, int S, const int* row_ptr, const int* col,
                                    const int* J, const int* h, cudaStream_t st);

}  // namespace isg
