// Random-number streams, state initialisation and the parallel-tempering pass.
#include <algorithm>
#include "ising_internal.cuh"
#include "split_math.cuh"

namespace isg {
namespace {

// ---------------------------------------------------------------- MT19937
// One block per stream.  x_w for w >= 624 follows x_w = x_{w-227} ^
// twist(x_{w-624}, x_{w-623}); the 227 words w in [B, B+227) depend only on
// words below B, so a block computes them in parallel.  The ring keeps the
// last 1024 words, so slot w & 1023 (written) never aliases a slot read in the
// same step (reads reach back 624 words at most).  Output j of the stream is
// temper(x_{624+j}).
__device__ __forceinline__ uint32_t mt_step_word(uint32_t* ring, unsigned long long w)
{
    const uint32_t x = mt_recur(ring[(w - 624) & (kMtRing - 1)], ring[(w - 623) & (kMtRing - 1)],
                                ring[(w - 227) & (kMtRing - 1)]);
    ring[w & (kMtRing - 1)] = x;
    return mt_temper(x);
}

// Sweep words are consumed column-major ([replica][position][slice]), but the
// stream produces them slice by slice.  Words of four consecutive slices are
// collected in shared memory and each column's 4-word block is then written
// with one 16-byte store; the per-step barriers therefore only wait on shared
// memory.  `group` words of the stream = 4 slices (fewer at the end of a
// sweep when M is not a multiple of 4).
constexpr int kGenGroupMaxS = 4096;  // slice sizes up to this use the staged path

__device__ __forceinline__ void mt_gen_body(const MtGenArgs& a, const int stream)
{
    extern __shared__ __align__(16) uint32_t gbuf[];  // [4][S] staged words, then [S] site positions
    __shared__ uint32_t ring[kMtRing];
    const bool swap = a.do_swap && stream == a.R;
    uint32_t* gring = a.ring + size_t(stream) * kMtRing;
    for (int i = threadIdx.x; i < kMtRing; i += blockDim.x)
        ring[i] = gring[i];
    const unsigned long long w0 = a.pos[stream];
    __syncthreads();

    long long nwords = a.nwords;
    if (swap) {
        // words of `swap_passes` passes starting at pass parity par0
        const int par0 = int(a.counters[1] & 1ull);
        const int n_even = a.R / 2;        // pairs (0,1),(2,3),...  = floor(R/2)
        const int n_odd = (a.R - 1) / 2;   // pairs (1,2),(3,4),...  = floor((R-1)/2)
        const int n_first = par0 ? n_odd : n_even;
        const int n_pair = n_even + n_odd;
        nwords = (long long)(a.swap_passes / 2) * n_pair + ((a.swap_passes & 1) ? n_first : 0);
        for (long long base = 0; base < nwords; base += kMtStep) {
            const long long cnt = min((long long)kMtStep, nwords - base);
            if (threadIdx.x < cnt) {
                const long long k = base + threadIdx.x;
                const uint32_t out = mt_step_word(ring, w0 + (unsigned long long)k);
                const long long cyc = k / n_pair, rem = k - cyc * n_pair;
                const long long prel = (rem < n_first) ? 2 * cyc : 2 * cyc + 1;
                const int j = int((rem < n_first) ? rem : rem - n_first);
                a.swbuf[size_t(prel) * a.maxpairs + j] = out;
            }
            __syncthreads();
        }
    } else if (a.mode == 1 || a.S > kGenGroupMaxS) {
        // initial spins, or slices too large to stage: direct stores
        for (long long base = 0; base < nwords; base += kMtStep) {
            const long long cnt = min((long long)kMtStep, nwords - base);
            if (threadIdx.x < cnt) {
                const long long k = base + threadIdx.x;
                const uint32_t out = mt_step_word(ring, w0 + (unsigned long long)k);
                if (a.mode == 1) {
                    a.spins[size_t(stream) * a.N + k] = (out >> 31) ? int8_t(1) : int8_t(-1);
                } else {
                    const long long c = k / a.N;
                    const int i = int(k - c * a.N);
                    const int t = i / a.S, q = i - t * a.S;
                    a.wbuf[size_t(c) * a.wbuf_sweep_stride +
                           (size_t(stream) * a.S + a.pos_of_site[q]) * a.Mp + t] = out;
                }
            }
            __syncthreads();
        }
    } else {
        const int S = a.S, M = a.M;
        uint32_t* spos = gbuf + 4 * S;  // [S] the column position of each site, staged once
        for (int q = threadIdx.x; q < S; q += blockDim.x)
            spos[q] = uint32_t(a.pos_of_site[q]);
        __syncthreads();
        const long long sweeps = nwords / a.N;
        // ring slots need only the low bits of the stream position: 32-bit
        // arithmetic (w & 1023 of a 64-bit w equals that of its low word)
        uint32_t wl = uint32_t(w0);
        for (long long c = 0; c < sweeps; ++c) {
            uint32_t* wsw = a.wbuf + size_t(c) * a.wbuf_sweep_stride + size_t(stream) * S * a.Mp;
            for (int t0 = 0; t0 < M; t0 += 4) {
                const int group = min(4, M - t0) * S;
                for (int base = 0; base < group; base += kMtStep) {
                    if (int(threadIdx.x) < min(kMtStep, group - base)) {
                        const int kk = base + threadIdx.x;
                        const uint32_t w = wl + uint32_t(kk);
                        const uint32_t x = mt_recur(ring[(w - 624u) & (kMtRing - 1)],
                                                    ring[(w - 623u) & (kMtRing - 1)],
                                                    ring[(w - 227u) & (kMtRing - 1)]);
                        ring[w & (kMtRing - 1)] = x;
                        gbuf[kk] = mt_temper(x);
                    }
                    __syncthreads();
                }
                // flush: column q gets words of slices t0..t0+3 as one 16-byte store
                for (int q = threadIdx.x; q < S; q += blockDim.x) {
                    const uint4 v = make_uint4(gbuf[q], gbuf[S + q], gbuf[2 * S + q], gbuf[3 * S + q]);
                    *reinterpret_cast<uint4*>(wsw + size_t(spos[q]) * a.Mp + t0) = v;
                }
                __syncthreads();
                wl += uint32_t(group);
            }
        }
    }
    for (int i = threadIdx.x; i < kMtRing; i += blockDim.x)
        gring[i] = ring[i];
    if (threadIdx.x == 0)
        a.pos[stream] = w0 + (unsigned long long)nwords;
}

__global__ void __launch_bounds__(256) mt_gen_kernel(const MtGenArgs a)
{
    mt_gen_body(a, a.first_stream + int(blockIdx.x));
}

// Batched: block b generates stream items[b].block of instance items[b].inst.
__global__ void __launch_bounds__(256) mt_gen_batch_kernel(const MtGenArgs* __restrict__ args,
                                                           const BatchItem* __restrict__ items)
{
    __shared__ MtGenArgs sa;
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0)
        sa = args[it.inst];
    __syncthreads();
    mt_gen_body(sa, it.block);
}

// ------------------------------------------------------------ Philox init
__global__ void philox_init_kernel(int8_t* spins, int R, int N, int S, uint32_t seed, uint32_t inst)
{
    const long long total = (long long)R * N;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = int(idx / N), i = int(idx - (long long)r * N);
        const int t = i / S, q = i - t * S;
        const uint4 ctr = make_uint4(uint32_t((t >> 2) * S + q), 0u, inst, 3u);
        const uint32_t u = pick4(philox4x32_10(ctr, seed, uint32_t(r)), t & 3);
        spins[idx] = (u >> 31) ? int8_t(1) : int8_t(-1);
    }
}

// ---------------------------------------------------- fields and energies
// f_i = h_i + sum_j J_ij s_j; E = -1/2 sum_i s_i (f_i + h_i) (each edge once).
template <typename FT>
__global__ void __launch_bounds__(256) state_init_kernel(const int8_t* spins, FT* fields, int* E,
                                                         int N, const int* row_ptr, const int* col,
                                                         const int* J, const int* h)
{
    __shared__ long long red[256];
    const int r = blockIdx.x;
    const int8_t* s = spins + size_t(r) * N;
    long long acc = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        int f = h[i];
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            f += J[e] * int(s[col[e]]);
        fields[size_t(r) * N + i] = FT(f);
        acc += (long long)s[i] * (f + h[i]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        E[r] = int(-red[0] / 2);
}

// Split couplings: f_i = h_i + sum over spatial j of J_ij s_j (j in the slice
// of i), E = -1/2 sum_i s_i (f_i + h_i) (each spatial edge once) and
// C = -1/2 sum_i s_i tau_i, tau_i the sum of the Trotter neighbours' spins
// (each Trotter pair once).
template <typename FT>
__global__ void __launch_bounds__(256) split_state_init_kernel(const int8_t* spins, FT* fields, int* E,
                                                               int* C, int N, int S, const int* row_ptr,
                                                               const int* col, const int* J,
                                                               const int* h)
{
    __shared__ long long red_e[256], red_c[256];
    const int r = blockIdx.x;
    const int8_t* s = spins + size_t(r) * N;
    long long acc_e = 0, acc_c = 0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int ti = i / S;
        int f = h[i], tau = 0;
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int j = col[e];
            if (j / S == ti)
                f += J[e] * int(s[j]);
            else
                tau += int(s[j]);
        }
        fields[size_t(r) * N + i] = FT(f);
        acc_e += (long long)s[i] * (f + h[i]);
        acc_c += (long long)s[i] * tau;
    }
    red_e[threadIdx.x] = acc_e;
    red_c[threadIdx.x] = acc_c;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red_e[threadIdx.x] += red_e[threadIdx.x + w];
            red_c[threadIdx.x] += red_c[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        E[r] = int(-red_e[0] / 2);
        C[r] = int(-red_c[0] / 2);
    }
}

// -------------------------------------------------------- PT pass
// Pass p tries pairs (k, k+1), k = 2j + (p & 1).  Pairs of one pass are
// disjoint, so each thread decides and applies its own pairs.
__device__ __forceinline__ void pt_body(const PtArgs& a)
{
    const unsigned long long p = a.counters[1];
    const int par = int(p & 1ull);
    const int npairs = par ? (a.R - 1) / 2 : a.R / 2;
    for (int j = threadIdx.x; j < npairs; j += blockDim.x) {
        const int k = 2 * j + par;
        const int sa = a.slot_of_temp[k], sb = a.slot_of_temp[k + 1];
        const long long d = (long long)a.E[sa] - (long long)a.E[sb];
        uint32_t u;
        if (a.rng == 0) {
            u = a.swbuf[size_t(a.pass_rel) * a.maxpairs + j];
        } else {
            const uint4 ctr = make_uint4(uint32_t(j) >> 2, uint32_t(p), a.inst, 1u);
            u = pick4(philox4x32_10(ctr, a.seed, 0xFFFFFFFFu), j & 3);
        }
        bool acc;
        if (a.split) {
            const long long dc = (long long)a.C[sa] - (long long)a.C[sb];
            const uint32_t th = split_detail::swap_threshold(a.dbeta[k], a.dK[k], d, dc);
            acc = th == 0xFFFFFFFFu || u < th;
        } else {
            acc = (d <= 0) || (d < a.swlen[k] && u < a.swthr[a.swoff[k] + d]);
        }
        if (acc) {
            a.slot_of_temp[k] = sb;
            a.slot_of_temp[k + 1] = sa;
            a.temp_of_slot[sa] = k + 1;
            a.temp_of_slot[sb] = k;
            a.swap_acc[k] += 1ull;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
        a.counters[1] = p + 1ull;
}

// int16 -> int32 widening of n fields (ising_read_state copies the result)
__global__ void __launch_bounds__(256) widen_i16_kernel(const int16_t* __restrict__ src, int* __restrict__ dst,
                                                        long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = int(src[i]);
}

__global__ void __launch_bounds__(1024) pt_kernel(const PtArgs a) { pt_body(a); }

// Batched: block b runs one PT pass of instance b.
__global__ void __launch_bounds__(1024) pt_batch_kernel(const PtArgs* __restrict__ args)
{
    __shared__ PtArgs sa;
    if (threadIdx.x == 0)
        sa = args[blockIdx.x];
    __syncthreads();
    pt_body(sa);
}

}  // namespace

cudaError_t launch_mt_gen(const MtGenArgs& a, int blocks, cudaStream_t st)
{
    // staged slices: 4 x S words (the kernel reads gbuf[2S + q], gbuf[3S + q]
    // even for a final group of fewer than 4 slices, so all 4S are allocated),
    // then the S site positions
    const size_t smem = (a.mode == 0 && a.S <= kGenGroupMaxS) ? 20u * a.S : 0u;
    mt_gen_kernel<<<blocks, 256, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mt_gen_set_smem_limit()
{
    cudaError_t e = cudaFuncSetAttribute(mt_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         20 * kGenGroupMaxS);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(mt_gen_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 20 * kGenGroupMaxS);
    return e;
}

cudaError_t launch_mt_gen_batch(const MtGenArgs* args, const BatchItem* items, int n_items,
                                int max_S, cudaStream_t st)
{
    const size_t smem = (max_S <= kGenGroupMaxS) ? 20u * size_t(max_S) : 0u;
    mt_gen_batch_kernel<<<n_items, 256, smem, st>>>(args, items);
    return cudaGetLastError();
}

cudaError_t launch_pt_batch(const PtArgs* args, int n_inst, int max_R, cudaStream_t st)
{
    int threads = ((max_R / 2 + 31) / 32) * 32;
    threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
    pt_batch_kernel<<<n_inst, threads, 0, st>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_philox_init(int8_t* spins, int R, int N, int S, uint32_t seed, uint32_t inst,
                               cudaStream_t st)
{
    const long long total = (long long)R * N;
    const int blocks = int(min((total + 255) / 256, 65535LL));
    philox_init_kernel<<<blocks, 256, 0, st>>>(spins, R, N, S, seed, inst);
    return cudaGetLastError();
}

cudaError_t launch_widen_i16(const int16_t* src, int* dst, long long n, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    const long long blocks = std::min<long long>((n + 255) / 256, 4096);
    widen_i16_kernel<<<int(blocks), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_state_init(const int8_t* spins, void* fields, int field_bits, int* E, int R,
                              int N, const int* row_ptr, const int* col, const int* J,
                              const int* h, cudaStream_t st)
{
    if (field_bits == 16)
        state_init_kernel<int16_t><<<R, 256, 0, st>>>(spins, static_cast<int16_t*>(fields), E, N,
                                                       row_ptr, col, J, h);
    else
        state_init_kernel<int32_t><<<R, 256, 0, st>>>(spins, static_cast<int32_t*>(fields), E, N,
                                                       row_ptr, col, J, h);
    return cudaGetLastError();
}

cudaError_t launch_split_state_init(const int8_t* spins, void* fields, int field_bits, int* E, int* C,
                                    int R, int N, int S, const int* row_ptr, const int* col,
                                    const int* J, const int* h, cudaStream_t st)
{
    if (field_bits == 16)
        split_state_init_kernel<int16_t><<<R, 256, 0, st>>>(spins, static_cast<int16_t*>(fields), E, C, N,
                                                             S, row_ptr, col, J, h);
    else
        split_state_init_kernel<int32_t><<<R, 256, 0, st>>>(spins, static_cast<int32_t*>(fields), E, C, N,
                                                             S, row_ptr, col, J, h);
    return cudaGetLastError();
}

cudaError_t launch_pt(const PtArgs& a, cudaStream_t st)
{
    const int npairs = a.R / 2;
    int threads = ((npairs + 31) / 32) * 32;
    threads = threads < 32 ? 32 : (threads > 1024 ? 1024 : threads);
    pt_kernel<<<1, threads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace isg
