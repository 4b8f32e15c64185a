// Register-resident wavefront sweep (M <= 32 slices, slice tables in shared
// memory), optionally running many sweeps with the parallel-tempering pass
// fused behind a bounded grid barrier.
//
// Same schedule and exactness argument as the generic kernel (sweep_impl.cuh):
// level(q, t) = lev0(q) + t, a barrier between levels.  What changes is where
// the per-column data lives.  A thread owns columns x = tid + c*T (x = p*G+g)
// and keeps, per column, in registers:
//   bits  the M spins of the column (bit t = spin (q, t) is +1); only the
//         owner reads or writes them, so the Trotter part of the field,
//         Jtau (s_{t-1} + s_{t+1}), costs two bit extractions;
//   cur   the four random words of the current block t>>2, and
//   nxt   the next block, fetched (MT19937, from the word buffer) or computed
//         (Philox) a few levels before it is needed, so neither the memory
//         latency nor the Philox rounds sit on the critical path of a level.
// The spatial part of every field stays in shared memory (fsp) because
// neighbours in other columns update it, through shared-memory atomics.
//
// Fused PT.  After every `swap_every` sweeps each block publishes the
// energies of its replicas, waits at a grid barrier (bounded: on timeout it
// raises the error flag and returns), and then every block performs the same
// PT pass on its own copy of the temperature labels, so no second barrier is
// needed.  Energies are published into one of two buffers by pass parity: a
// block can only overwrite a buffer after every block has passed the next
// barrier, i.e. after everybody finished reading it.
#pragma once
#include <climits>

#include "field_ops.cuh"
#include "ising_internal.cuh"

namespace isg {
namespace fast_detail {

struct FastLayout {
    uint32_t nbr_off, nbr, jtau, pos, site, fsp, thr, eacc, colw, slot, temp, total;
};

__host__ __device__ inline FastLayout fast_layout(const SweepArgs& a, int fbytes)
{
    FastLayout L{};
    uint32_t o = 16;  // mbarrier
    L.nbr_off = o; o += r16(4u * (a.S + 1));
    L.nbr = o;     o += r16(4u * (a.nbr_count > 0 ? a.nbr_count : 1));
    L.jtau = o;    o += r16(4u * a.S);
    L.pos = o;     o += r16(4u * a.S);
    L.site = o;    o += r16(4u * a.S);
    // with MT19937 the lean kernel reuses the table region, once the tables
    // are unpacked into registers, to stage two 16-byte word blocks per column
    if (a.rng == 0 && o < 16u + 32u * a.S)
        o = 16u + 32u * a.S;
    L.fsp = o;     o += r16(uint32_t(fbytes) * a.N * a.G);
    L.thr = o;     o += r16(4u * a.G * a.K);
    L.eacc = o;    o += r16(4u * a.G);
    // long columns (M > 32, lean kernel only): M / 32 words per column
    L.colw = o;
    if (a.M > 32)
        o += r16(4u * uint32_t(a.S) * uint32_t(a.M / 32));
    if (a.swap_every > 0) {
        L.slot = o; o += r16(4u * a.R);
        L.temp = o; o += r16(4u * a.R);
    }
    L.total = o;
    return L;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier on a monotone arrival counter.  Returns false in every
// thread of the block when the wait gave up (error flag raised).
__device__ __forceinline__ bool grid_sync(unsigned* ctr, unsigned target, int* err, int* s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr, 1u);
        int ok = 1;
        long long polls = 0;
        while (ld_acquire_gpu(ctr) < target) {
            if (++polls > (1LL << 22)) {
                ok = 0;
                set_err(err, kErrTimeout);
                break;
            }
            __nanosleep(64);
        }
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// Trotter field from the owner's column bits (M <= 32).
__device__ __forceinline__ int trotter_bits(uint32_t bits, int t, int M, int jt)
{
    if (M >= 3) {
        const int tm = (t == 0) ? M - 1 : t - 1;
        const int tp = (t == M - 1) ? 0 : t + 1;
        return jt * (2 * int(((bits >> tm) & 1u) + ((bits >> tp) & 1u)) - 2);
    }
    if (M == 2)
        return jt * (2 * int((bits >> (1 - t)) & 1u) - 1);
    return 0;
}

template <int RNG>
__device__ __forceinline__ uint4 rng_block(const SweepArgs& a, const uint32_t* wsw, int rg, int p,
                                           int q, int b, uint32_t sid)
{
    if (RNG == 0) {
        return __ldg(reinterpret_cast<const uint4*>(wsw + (size_t(rg) * a.S + p) * a.Mp) + b);
    } else {
        return philox4x32_10(make_uint4(uint32_t(b * a.S + q), sid, a.inst, 0u), a.seed, uint32_t(rg));
    }
}

// Register budget: columns per thread x ~12 registers must fit, so wider
// ownership caps the block size (1024 threads -> 64 registers per thread).
__host__ __device__ constexpr int fast_max_threads(int cmax)
{
    return cmax <= 2 ? 1024 : (cmax == 4 ? 512 : 256);
}

// Body of one block: `blk` is the block's index within its instance and
// `nblk` the instance's number of blocks (the grid size for a single instance).
template <typename FT, int RNG, int CMAX>
__device__ __forceinline__ void fast_body(const SweepArgs& a, const int blk, const int nblk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const FastLayout L = fast_layout(a, Fsp<FT>::kBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const int T = blockDim.x, tid = threadIdx.x;
    const int S = a.S, M = a.M, N = a.N, G = a.G, K = a.K, R = a.R;
    const int r0 = blk * G;
    const int Gb = min(G, R - r0);
    const int* nbr_off = reinterpret_cast<const int*>(smem + L.nbr_off);
    const uint32_t* nbr = reinterpret_cast<const uint32_t*>(smem + L.nbr);
    const int* jtau = reinterpret_cast<const int*>(smem + L.jtau);
    const int* pos = reinterpret_cast<const int*>(smem + L.pos);
    const int* site = reinterpret_cast<const int*>(smem + L.site);
    void* fsp = smem + L.fsp;
    uint32_t* thr_s = reinterpret_cast<uint32_t*>(smem + L.thr);
    int* eacc = reinterpret_cast<int*>(smem + L.eacc);
    int* slot_s = reinterpret_cast<int*>(smem + L.slot);
    int* temp_s = reinterpret_cast<int*>(smem + L.temp);
    const bool fused = a.swap_every > 0;

    // ---- stage the slice tables with bulk copies
    if (tid == 0)
        mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
        const uint32_t b0 = r16(4u * (S + 1)), b1 = r16(4u * (a.nbr_count > 0 ? a.nbr_count : 1));
        const uint32_t b2 = r16(4u * S);
        mbar_expect_tx(bar, b0 + b1 + 3 * b2);
        bulk_g2s(smem + L.nbr_off, a.nbr_off, b0, bar);
        bulk_g2s(smem + L.nbr, a.nbr, b1, bar);
        bulk_g2s(smem + L.jtau, a.jtau, b2, bar);
        bulk_g2s(smem + L.pos, a.pos, b2, bar);
        bulk_g2s(smem + L.site, a.site, b2, bar);
    }
    for (int i = tid; i < G; i += T)
        eacc[i] = 0;
    if (fused)
        for (int i = tid; i < R; i += T) {
            slot_s[i] = a.slot_of_temp[i];
            temp_s[i] = a.temp_of_slot[i];
        }
    if (tid == 0)
        s_flag = mbar_wait(bar, 0, kWaitPolls) ? 1 : 0;
    __syncthreads();
    if (!s_flag) {
        if (tid == 0)
            set_err(a.err, kErrTimeout);
        return;
    }
    mbar_wait(bar, 0, kWaitPolls);  // phase complete: per-thread acquire of the tables

    // ---- spatial fields f_sp = f - Jtau (s_{t-1} + s_{t+1}), coalesced over i
    for (int g = 0; g < Gb; ++g) {
        const int8_t* sp = a.spins + size_t(r0 + g) * N;
        const FT* fg = static_cast<const FT*>(a.fields) + size_t(r0 + g) * N;
        for (int i = tid; i < N; i += T) {
            const int t = i / S, q = i - t * S, p = pos[q];
            int ft = 0;
            if (M >= 3) {
                const int tm = (t == 0) ? M - 1 : t - 1, tp = (t == M - 1) ? 0 : t + 1;
                ft = jtau[p] * (int(sp[tm * S + q]) + int(sp[tp * S + q]));
            } else if (M == 2) {
                ft = jtau[p] * int(sp[(1 - t) * S + q]);
            }
            Fsp<FT>::st(fsp, (p * M + t) * G + g, int(fg[i]) - ft);
        }
    }
    for (int idx = tid; idx < Gb * K; idx += T) {
        const int g = idx / K, k = idx - g * K;
        const int temp = fused ? temp_s[r0 + g] : a.temp_of_slot[r0 + g];
        thr_s[idx] = a.thr[size_t(temp) * K + k];
    }

    // ---- owned columns: registers
    const int g = tid & (G - 1);
    const bool live = g < Gb;
    const int rg = r0 + g;
    const int SG = S * G;
    int lv[CMAX], jt[CMAX], eb[CMAX];
    uint32_t bits[CMAX];
    uint4 cur[CMAX], nxt[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        const int x = tid + c * T;
        lv[c] = INT_MAX / 2;
        jt[c] = 0;
        eb[c] = 0;
        bits[c] = 0u;
        cur[c] = nxt[c] = make_uint4(0u, 0u, 0u, 0u);
        if (live && x < SG) {
            const int p = x >> a.lg_G;
            lv[c] = a.lev0[p];
            jt[c] = jtau[p];
            eb[c] = (nbr_off[p] << 8) | (nbr_off[p + 1] - nbr_off[p]);
            const int8_t* sp = a.spins + size_t(rg) * N + site[p];
            uint32_t b = 0u;
            for (int t = 0; t < M; ++t)
                b |= (sp[size_t(t) * S] > 0 ? 1u : 0u) << t;
            bits[c] = b;
        }
    }
    __syncthreads();

    const unsigned long long sweep0 = a.counters[0];
    const unsigned long long pass0 = a.counters[1];
    const int nrb = (M + 3) >> 2;  // random-word blocks per column
    int npass = 0;
    int dE = 0;

    for (int sw = 0; sw < a.nsweeps; ++sw) {
        const uint32_t sid = uint32_t(sweep0 + sw);
        const uint32_t* wsw = (RNG == 0) ? a.wbuf + size_t(sw) * a.wbuf_sweep_stride : nullptr;
        const uint32_t* thr_g = thr_s + g * K;
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
            if (lv[c] < INT_MAX / 2) {
                const int p = (tid + c * T) >> a.lg_G;
                const int q = (RNG == 1) ? site[p] : 0;
                cur[c] = rng_block<RNG>(a, wsw, rg, p, q, 0, sid);
                if (RNG == 0 && nrb > 1)
                    nxt[c] = rng_block<RNG>(a, wsw, rg, p, q, 1, sid);
            }
        }
        for (int l = 0; l < a.D; ++l) {
#pragma unroll
            for (int c = 0; c < CMAX; ++c) {
                const int t = l - lv[c];
                if (unsigned(t) < unsigned(M)) {
                    const int p = (tid + c * T) >> a.lg_G;
                    if (t > 0 && (t & 3) == 0) {
                        cur[c] = nxt[c];
                        if (RNG == 0 && (t >> 2) + 1 < nrb)
                            nxt[c] = rng_block<RNG>(a, wsw, rg, p, 0, (t >> 2) + 1, sid);
                    }
                    const int fidx = (p * M + t) * G + g;
                    const int fs = Fsp<FT>::ld(fsp, fidx);
                    const uint32_t bw = bits[c];
                    const int s = 2 * int((bw >> t) & 1u) - 1;
                    const int k = s * (fs + trotter_bits(bw, t, M, jt[c]));
                    const uint32_t u = pick4(cur[c], t & 3);
                    const bool acc = (k <= 0) || (k < K && u < thr_g[k]);
                    if (acc) {
                        bits[c] = bw ^ (1u << t);
                        dE += 2 * k;
                        const int m2s = -2 * s;
                        const int e0 = eb[c] >> 8, ne = eb[c] & 0xFF;
                        for (int e = 0; e < ne; ++e) {
                            const uint32_t en = nbr[e0 + e];
                            Fsp<FT>::add(fsp, (int(en >> 16) * M + t) * G + g,
                                         m2s * int(int16_t(en & 0xFFFFu)));
                        }
                    }
                    if (RNG == 1 && (t & 3) == 1 && (t >> 2) + 1 < nrb)
                        nxt[c] = rng_block<RNG>(a, wsw, rg, p, site[p], (t >> 2) + 1, sid);
                }
            }
            __syncthreads();
        }

        if (fused && (sw + 1) % a.swap_every == 0) {
            // publish energies, meet at the grid barrier, run the PT pass
            if (live && dE != 0)
                atomicAdd(&eacc[g], dE);
            dE = 0;
            __syncthreads();
            int* Ep = a.E_pub + size_t(npass & 1) * R;
            if (tid < Gb) {
                const int e = a.E[r0 + tid] + eacc[tid];
                a.E[r0 + tid] = e;
                Ep[r0 + tid] = e;
                eacc[tid] = 0;
            }
            if (nblk == 1)  // a one-block instance has nobody else to wait for
                __syncthreads();
            else if (!grid_sync(a.gridbar, unsigned(npass + 1) * unsigned(nblk), a.err, &s_flag))
                return;
            if (tid < 32) {
                const unsigned long long p = pass0 + npass;
                const int par = int(p & 1ull);
                const int npairs = par ? (R - 1) / 2 : R / 2;
                for (int j = tid; j < npairs; j += 32) {
                    const int k = 2 * j + par;
                    const int sa = slot_s[k], sb = slot_s[k + 1];
                    const long long d = (long long)__ldcg(Ep + sa) - (long long)__ldcg(Ep + sb);
                    uint32_t u;
                    if (RNG == 0)
                        u = a.swbuf[size_t(npass) * a.maxpairs + j];
                    else
                        u = pick4(philox4x32_10(make_uint4(uint32_t(j) >> 2, uint32_t(p), a.inst, 1u),
                                                a.seed, 0xFFFFFFFFu), j & 3);
                    if ((d <= 0) || (d < a.swlen[k] && u < a.swthr[a.swoff[k] + d])) {
                        slot_s[k] = sb;
                        slot_s[k + 1] = sa;
                        temp_s[sa] = k + 1;
                        temp_s[sb] = k;
                        if (blk == 0)
                            a.swap_acc[k] += 1ull;
                    }
                }
            }
            __syncthreads();
            for (int idx = tid; idx < Gb * K; idx += T) {
                const int gg = idx / K, k = idx - gg * K;
                thr_s[idx] = a.thr[size_t(temp_s[r0 + gg]) * K + k];
            }
            __syncthreads();
            ++npass;
        }
    }

    // ---- energies and write-back of the owned columns
    if (live && dE != 0)
        atomicAdd(&eacc[g], dE);
    __syncthreads();
    if (tid < Gb)
        a.E[r0 + tid] += eacc[tid];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        if (lv[c] < INT_MAX / 2) {
            const int p = (tid + c * T) >> a.lg_G;
            const int q = site[p];
            int8_t* sp = a.spins + size_t(rg) * N + q;
            FT* fg = static_cast<FT*>(a.fields) + size_t(rg) * N + q;
            for (int t = 0; t < M; ++t) {
                sp[size_t(t) * S] = ((bits[c] >> t) & 1u) ? int8_t(1) : int8_t(-1);
                fg[size_t(t) * S] =
                    FT(Fsp<FT>::ld(fsp, (p * M + t) * G + g) + trotter_bits(bits[c], t, M, jt[c]));
            }
        }
    }
    if (fused && blk == 0)
        for (int i = tid; i < R; i += T) {
            a.slot_of_temp[i] = slot_s[i];
            a.temp_of_slot_out[i] = temp_s[i];
        }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done_blocks, 1u);
        if (prev == unsigned(nblk) - 1u) {
            a.counters[0] += (unsigned long long)a.nsweeps;
            a.counters[1] += (unsigned long long)npass;
            *a.done_blocks = 0u;
            __threadfence();
        }
    }
}

template <typename FT, int RNG, int CMAX>
__global__ void __launch_bounds__(fast_max_threads(CMAX), 1) fast_kernel(const SweepArgs a)
{
    fast_body<FT, RNG, CMAX>(a, int(blockIdx.x), int(gridDim.x));
}

// Batched launch over many instances: each block copies its instance's
// arguments into shared memory (so that every later read is a shared load).
template <typename FT, int RNG, int CMAX>
__global__ void __launch_bounds__(fast_max_threads(CMAX), 1)
    fast_batch_kernel(const SweepArgs* __restrict__ args, const BatchItem* __restrict__ items)
{
    __shared__ SweepArgs sa;
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0)
        sa = args[it.inst];
    __syncthreads();
    fast_body<FT, RNG, CMAX>(sa, it.block, sa.inst_blocks);
}

template <typename FT, int RNG>
void* pick_fast(int cmax, bool batch = false)
{
    switch (cmax) {
    case 1: return batch ? reinterpret_cast<void*>(&fast_batch_kernel<FT, RNG, 1>)
                   : reinterpret_cast<void*>(&fast_kernel<FT, RNG, 1>);
    case 2: return batch ? reinterpret_cast<void*>(&fast_batch_kernel<FT, RNG, 2>)
                   : reinterpret_cast<void*>(&fast_kernel<FT, RNG, 2>);
    case 4: return batch ? reinterpret_cast<void*>(&fast_batch_kernel<FT, RNG, 4>)
                   : reinterpret_cast<void*>(&fast_kernel<FT, RNG, 4>);
    case 8: return batch ? reinterpret_cast<void*>(&fast_batch_kernel<FT, RNG, 8>)
                   : reinterpret_cast<void*>(&fast_kernel<FT, RNG, 8>);
    default: return nullptr;
    }
}

}  // namespace fast_detail

void* fast_kernel_i16(int rng, int cmax, bool batch = false);
void* fast_kernel_i32(int rng, int cmax, bool batch = false);

}  // namespace isg
