// Lean register-resident wavefront sweep for the layered models of the
// paper's QMC setting: one replica per block, M in {4, 8, 16, 32} slices (or,
// as the LONG instantiation, any multiple of 32 up to 1024: see below),
// spatial degree <= 6 and |J| <= 63.  Same schedule, state and fused-PT
// protocol as fast_impl.cuh (level(q, t) = lev0(q) + t; spatial fields in
// shared memory with atomic neighbour updates; column bits and random-word
// blocks in registers); the item path is cut to what the decision needs:
//
//  * Column bits are kept replicated across the 32-bit word (period M), so a
//    single funnel-shift rotation by t-1 brings s_{t-1}, s_t, s_{t+1} (ring
//    wrap included) to bits 0..2.
//  * The neighbour list of each owned column is unpacked once into registers
//    as (32-bit field word of slice 0, 2J), fully unrolled (spatial degree
//    <= 6: the 4 lattice neighbours plus two matchings); with M even the
//    half-word parity of every neighbour's field equals t's parity, so one
//    shift per item serves all neighbours (int16 fields).  Missing
//    neighbours are padded with a zero delta aimed at the item's own field
//    word (no other item of the level touches it), so the six atomics are
//    issued unconditionally once the flip is accepted.
//  * Random words come in blocks of four (t>>2): block b+1 is fetched or
//    computed while block b is consumed.  MT19937 words are staged global ->
//    shared with cp.async, two blocks per column: a barrier must wait for a
//    warp's outstanding register loads, but not for its asynchronous copies,
//    so the staging latency never lands on a level.  Philox: the ten rounds
//    of block b+1 are spread over the four levels of block b (one state per
//    thread: the block size is at least the widest level, so a thread has at
//    most one busy column per level).
//  * With at most 32 tabulated thresholds, lane k of every warp holds T[k] and
//    the lookup of T[k] is a warp shuffle in a converged section.
//  * LONG (M = 32 KW, KW >= 2): the column lives as KW words in shared
//    memory; a thread holds the word of its busy slice and the words before
//    and after it (ring order), so s_{t-1}, s_t, s_{t+1} are register bits.
//    When the slice leaves a word, the word is stored and the next-but-one is
//    loaded, 32 levels before it is needed; the words of slices 0 and M - 1
//    are stored before the other end of the ring reads them.
//  * SPLIT (split couplings, ising_set_trotter): the global fields are the
//    spatial ones, the Trotter coupling of the graph is ignored, and a flip
//    looks up the temperature's table at (k_s, k_tau), k_s = s f_space and
//    k_tau = s (s_{t-1} + s_{t+1}); the block accumulates the spatial energy
//    and the Trotter sum C apart, and the fused PT pass evaluates
//    z = dbeta dE + dK dC with the deterministic exponential (split_math.cuh).
#pragma once
#include <climits>

#include "fast_impl.cuh"
#include "split_math.cuh"

namespace isg {
namespace lean_detail {

using fast_detail::FastLayout;
using fast_detail::fast_layout;
using fast_detail::grid_sync;
using fast_detail::rng_block;

constexpr int kMaxDeg = 6;

__host__ __device__ constexpr int lean_max_threads(int cmax)
{
    return cmax <= 1 ? 1024 : (cmax == 2 ? 512 : 256);
}

// two resident blocks of 256 threads per SM for 4 columns per thread (128
// registers each): a 256-replica ladder then fits on the GPU at once
__host__ __device__ constexpr int lean_min_blocks(int cmax) { return cmax == 4 ? 2 : 1; }

// The small-block instantiation (two columns per thread, at most
// kLeanSmallThreads = 128 threads) for ladders of many small replicas, where
// residency rather than the length of one level bounds the throughput:
// twelve resident blocks per SM with MT19937 words (at most 42 registers a
// thread; 1.17e11 attempts/s on 4096 spins x 65536 replicas against 1.11e11
// with eight), eight with Philox (at most 64 registers: the ten rounds spill
// at twelve, 1.08e11 against 1.22e11).
__host__ __device__ constexpr int lean_bound_threads(int cmax, bool small)
{
    return small ? kLeanSmallThreads : lean_max_threads(cmax);
}
__host__ __device__ constexpr int lean_bound_blocks(int cmax, bool small, int rng, bool split = false)
{
    return small ? (rng == 0 && !split ? 12 : 8) : lean_min_blocks(cmax);
}

// Body of one block: `blk` is the replica (block) index within its instance
// and `nblk` the instance's number of blocks (the grid size for one instance).
template <typename FT, int RNG, int CMAX, bool LONG, bool SPLIT = false>
__device__ __forceinline__ void lean_body(const SweepArgs& a, const int blk, const int nblk)
{
    constexpr bool kI16 = sizeof(FT) == 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const FastLayout L = fast_layout(a, Fsp<FT>::kBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const int T = blockDim.x, tid = threadIdx.x;
    const int S = a.S, M = a.M, N = a.N, K = a.K, R = a.R;
    const int r = blk;  // one replica per block
    const int* nbr_off = reinterpret_cast<const int*>(smem + L.nbr_off);
    const uint32_t* nbr = reinterpret_cast<const uint32_t*>(smem + L.nbr);
    const int* jtau = reinterpret_cast<const int*>(smem + L.jtau);
    const int* pos = reinterpret_cast<const int*>(smem + L.pos);
    const int* site = reinterpret_cast<const int*>(smem + L.site);
    void* fsp = smem + L.fsp;
    unsigned* fsw = reinterpret_cast<unsigned*>(smem + L.fsp);
    uint32_t* colw = reinterpret_cast<uint32_t*>(smem + L.colw);  // LONG: [S][M / 32] column words
    const int KW = M >> 5;                                          // LONG: words per column
    uint32_t* thr_s = reinterpret_cast<uint32_t*>(smem + L.thr);
    int* eacc = reinterpret_cast<int*>(smem + L.eacc);
    int* slot_s = reinterpret_cast<int*>(smem + L.slot);
    int* temp_s = reinterpret_cast<int*>(smem + L.temp);
    const bool fused = a.swap_every > 0;

    // ---- stage tables (bulk copies), labels, spatial fields, thresholds
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
    if (tid == 0) {
        eacc[0] = 0;
        if constexpr (SPLIT)
            eacc[1] = 0;  // the region holds 16 bytes even for one replica
    }
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
    mbar_wait(bar, 0, kWaitPolls);
    {
        const int8_t* sp = a.spins + size_t(r) * N;
        const FT* fg = static_cast<const FT*>(a.fields) + size_t(r) * N;
        for (int i = tid; i < N; i += T) {
            const int t = i / S, q = i - t * S, p = pos[q];
            const int tm = (t == 0) ? M - 1 : t - 1, tp = (t == M - 1) ? 0 : t + 1;
            // SPLIT: the global fields already hold the spatial part only
            const int ft = SPLIT ? 0 : jtau[p] * (int(sp[tm * S + q]) + int(sp[tp * S + q]));
            Fsp<FT>::st(fsp, p * M + t, int(fg[i]) - ft);
        }
    }
    {
        const int temp = fused ? temp_s[r] : a.temp_of_slot[r];
        for (int k = tid; k < K; k += T)
            thr_s[k] = a.thr[size_t(temp) * K + k];
    }

    // ---- owned columns
    const uint32_t rep = (M == 32) ? 1u : (M == 16 ? 0x00010001u : (M == 8 ? 0x01010101u : 0x11111111u));
    int lv[CMAX], jd[CMAX], fb[CMAX];
    uint32_t bits[CMAX];  // M <= 32: the column, replicated with period M
    // LONG: the words k - 1, k, k + 1 (mod M / 32) around the word k of the
    // column's busy slice; a word is stored to `colw` when the slice leaves it
    uint32_t cwP[CMAX], cwW[CMAX], cwN[CMAX];
    uint32_t nb[CMAX][kMaxDeg];
    uint4 ba[CMAX];  // Philox: the current word block of each column
    unsigned char* stage = smem + L.nbr_off;  // MT19937: [S][2 blocks][16 B]
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        const int p = tid + c * T;
        lv[c] = INT_MAX / 2;
        jd[c] = 0;
        fb[c] = 0;
        bits[c] = 0u;
        cwP[c] = cwW[c] = cwN[c] = 0u;
        ba[c] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int e = 0; e < kMaxDeg; ++e)
            nb[c][e] = 0u;
        if (p < S) {
            lv[c] = a.lev0[p];
            const int e0 = nbr_off[p], deg = nbr_off[p + 1] - e0;
            jd[c] = ((SPLIT ? 0 : jtau[p]) << 8) | deg;  // SPLIT: no Trotter part in the field
            fb[c] = p * M;
            const uint32_t own = kI16 ? uint32_t(p * M / 2) : uint32_t(p * M);
#pragma unroll
            for (int e = 0; e < kMaxDeg; ++e) {
                nb[c][e] = own << 8;  // padding: zero delta on the own field word
                if (e < deg) {
                    const uint32_t en = nbr[e0 + e];
                    const int q2 = int(en >> 16);
                    const int twoJ = 2 * int(int16_t(en & 0xFFFFu));
                    const uint32_t word = kI16 ? uint32_t(q2 * M / 2) : uint32_t(q2 * M);
                    nb[c][e] = (word << 8) | (uint32_t(twoJ) & 0xFFu);
                }
            }
            const int8_t* sp = a.spins + size_t(r) * N + site[p];
            if constexpr (LONG) {
                for (int w = 0; w < KW; ++w) {
                    uint32_t b = 0u;
                    for (int i = 0; i < 32; ++i)
                        b |= (sp[size_t(32 * w + i) * S] > 0 ? 1u : 0u) << i;
                    colw[p * KW + w] = b;
                }
            } else {
                uint32_t b = 0u;
                for (int t = 0; t < M; ++t)
                    b |= (sp[size_t(t) * S] > 0 ? 1u : 0u) << t;
                bits[c] = b * rep;  // replicate the column with period M
            }
        }
    }
    __syncthreads();  // tables consumed: with MT19937 their region becomes `stage`

    const unsigned long long sweep0 = a.counters[0];
    const unsigned FULL = 0xFFFFFFFFu;
    const bool shfl_thr = !SPLIT && K <= 32;
    uint32_t thr_lane = (shfl_thr && (tid & 31) < K) ? thr_s[tid & 31] : 0u;
    const unsigned long long pass0 = a.counters[1];
    const int nrb = (M + 3) >> 2;  // random-word blocks per column
    int npass = 0;
    int dE = 0;
    int dC = 0;  // SPLIT: change of the Trotter sum C
    // Philox block in progress: one per thread, as a thread has at most one busy
    // column per level (the host sizes the block to the widest level)
    uint4 pc = make_uint4(0u, 0u, 0u, 0u);
    uint32_t pk0 = 0u, pk1 = 0u;

    for (int sw = 0; sw < a.nsweeps; ++sw) {
        const uint32_t sid = uint32_t(sweep0 + sw);
        const uint32_t* wsw = (RNG == 0) ? a.wbuf + size_t(sw) * a.wbuf_sweep_stride : nullptr;
#pragma unroll
        for (int c = 0; c < CMAX; ++c) {
            if (lv[c] < INT_MAX / 2) {
                const int p = tid + c * T;
                if constexpr (LONG) {  // slice 0 lies in word 0; slice M - 1 in the last word
                    cwP[c] = colw[p * KW + KW - 1];
                    cwW[c] = colw[p * KW];
                    cwN[c] = colw[p * KW + 1];
                }
                if (RNG == 0) {
                    const uint32_t* src = wsw + (size_t(r) * S + p) * a.Mp;
                    cp_async16(stage + p * 32, src);
                    if (nrb > 1)
                        cp_async16(stage + p * 32 + 16, src + 4);
                } else {
                    ba[c] = rng_block<RNG>(a, wsw, r, p, site[p], 0, sid);  // later blocks: see pc
                }
            }
        }
        for (int l = 0; l < a.D; ++l) {
#pragma unroll
            for (int c = 0; c < CMAX; ++c) {
                const int t0 = l - lv[c];
                const bool act = unsigned(t0) < unsigned(M);
                if (__any_sync(FULL, act)) {
                    // converged section: every lane runs it, inactive lanes on slice 0
                    const int t = act ? t0 : 0;
                    const int p = act ? tid + c * T : 0;  // inactive lanes address column 0
                    const int odd = (t >> 2) & 1;
                    if (RNG == 0 && act && (t & 3) == 0)
                        cp_async_wait_all();  // block t>>2 has landed in `stage`
                    const int fs = Fsp<FT>::ld(fsp, act ? fb[c] + t : 0);
                    if (RNG != 0 && act && (t & 3) == 0 && t > 0)
                        ba[c] = pc;  // block t>>2, finished over the previous four levels
                    const uint32_t u = (RNG == 0)
                        ? *reinterpret_cast<const uint32_t*>(stage + p * 32 + odd * 16 + (t & 3) * 4)
                        : pick4(ba[c], t & 3);
                    // bits 0, 1, 2 = s_{t-1}, s_t, s_{t+1} (ring wrap included)
                    uint32_t w3;
                    if constexpr (LONG) {
                        const int tb = t & 31;
                        const uint32_t sm1 = tb ? (cwW[c] >> (tb - 1)) : (cwP[c] >> 31);
                        const uint32_t sp1 = tb < 31 ? (cwW[c] >> (tb + 1)) : cwN[c];
                        w3 = (sm1 & 1u) | (((cwW[c] >> tb) & 1u) << 1) | ((sp1 & 1u) << 2);
                    } else {
                        w3 = __funnelshift_r(bits[c], bits[c], (t - 1) & 31);
                    }
                    const int s = 2 * int((w3 >> 1) & 1u) - 1;
                    const int ft = (jd[c] >> 8) * (2 * int((w3 & 1u) + ((w3 >> 2) & 1u)) - 2);
                    const int k = s * (fs + ft);
                    uint32_t tk;
                    bool take;
                    int kt = 0;
                    if constexpr (SPLIT) {
                        // k = k_s (ft = 0); entry (k_s + KS) * 3 + k_tau / 2 + 1, held inside
                        // the table for the idle lanes of the converged section
                        kt = s * (2 * int((w3 & 1u) + ((w3 >> 2) & 1u)) - 2);
                        const int idx = min(max((k + a.split_ks) * 3 + (kt >> 1) + 1, 0), K - 1);
                        tk = thr_s[idx];
                        take = act && (tk == 0xFFFFFFFFu || u < tk);
                    } else {
                        if (shfl_thr)
                            tk = __shfl_sync(FULL, thr_lane, (k > 0 && k < K) ? k : 0);
                        else
                            tk = (k > 0 && k < K) ? thr_s[k] : 0u;
                        take = act && ((k <= 0) || (k < K && u < tk));
                    }
                    if (take) {
                        if constexpr (LONG)
                            cwW[c] ^= 1u << (t & 31);
                        else
                            bits[c] ^= rep << t;
                        dE += 2 * k;
                        if constexpr (SPLIT)
                            dC += 2 * kt;
                        const int tw = kI16 ? (t >> 1) : t;
                        const int sh = kI16 ? ((t & 1) << 4) : 0;
#pragma unroll
                        for (int e = 0; e < kMaxDeg; ++e) {
                            const uint32_t v = nb[c][e];
                            const int d = -s * int(int8_t(v & 0xFFu));
                            atomicAdd(fsw + (v >> 8) + tw, unsigned(d) << sh);
                        }
                    }
                    if constexpr (LONG) {
                        if (act && (t & 31) == 31) {  // the slice leaves word k: store it, rotate
                            const int k = t >> 5;
                            colw[p * KW + k] = cwW[c];
                            if (k + 1 < KW) {
                                cwP[c] = cwW[c];
                                cwW[c] = cwN[c];
                                const int k2 = k + 2 < KW ? k + 2 : k + 2 - KW;
                                cwN[c] = colw[p * KW + k2];
                            }
                        }
                    }
                    if (RNG == 0) {
                        // block (t>>2)+1 replaces block (t>>2)-1 in the idle slot
                        if (act && (t & 3) == 0 && (t >> 2) + 1 < nrb && t > 0)
                            cp_async16(stage + p * 32 + (odd ^ 1) * 16, wsw + (size_t(r) * S + p) * a.Mp + t + 4);
                    } else if (act && (t >> 2) + 1 < nrb) {
                        // Philox: the ten rounds of block (t>>2)+1 spread over the four
                        // levels of block t>>2 (3, 3, 3, 1), so no level carries a whole
                        // call; the state is the thread's (one busy column per level)
                        const int ph = t & 3;
                        if (ph == 0) {
                            pc = make_uint4(uint32_t(((t >> 2) + 1) * S + site[p]), sid, a.inst, 0u);
                            pk0 = a.seed;
                            pk1 = uint32_t(r);
                        }
#pragma unroll
                        for (int i = 0; i < 3; ++i)
                            if (3 * ph + i < 10) {
                                const uint32_t lo0 = 0xD2511F53u * pc.x, hi0 = __umulhi(0xD2511F53u, pc.x);
                                const uint32_t lo1 = 0xCD9E8D57u * pc.z, hi1 = __umulhi(0xCD9E8D57u, pc.z);
                                pc = make_uint4(hi1 ^ pc.y ^ pk0, lo1, hi0 ^ pc.w ^ pk1, lo0);
                                pk0 += 0x9E3779B9u;
                                pk1 += 0xBB67AE85u;
                            }
                    }
                }
            }
            __syncthreads();
        }

        if (fused && (sw + 1) % a.swap_every == 0) {
            if (dE != 0)
                atomicAdd(&eacc[0], dE);
            dE = 0;
            if constexpr (SPLIT) {
                if (dC != 0)
                    atomicAdd(&eacc[1], dC);
                dC = 0;
            }
            __syncthreads();
            int* Ep = a.E_pub + size_t(npass & 1) * R;
            int* Cp = SPLIT ? a.C_pub + size_t(npass & 1) * R : nullptr;
            if (tid == 0) {
                const int e = a.E[r] + eacc[0];
                a.E[r] = e;
                Ep[r] = e;
                eacc[0] = 0;
                if constexpr (SPLIT) {
                    const int cs = a.C[r] + eacc[1];
                    a.C[r] = cs;
                    Cp[r] = cs;
                    eacc[1] = 0;
                }
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
                    bool take;
                    if constexpr (SPLIT) {
                        const long long dc = (long long)__ldcg(Cp + sa) - (long long)__ldcg(Cp + sb);
                        const uint32_t th = split_detail::swap_threshold(a.dbeta[k], a.dK[k], d, dc);
                        take = th == 0xFFFFFFFFu || u < th;
                    } else {
                        take = (d <= 0) || (d < a.swlen[k] && u < a.swthr[a.swoff[k] + d]);
                    }
                    if (take) {
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
            for (int k = tid; k < K; k += T)
                thr_s[k] = a.thr[size_t(temp_s[r]) * K + k];
            __syncthreads();
            thr_lane = (shfl_thr && (tid & 31) < K) ? thr_s[tid & 31] : 0u;
            ++npass;
        }
    }

    // ---- energies and write-back of the owned columns
    if (dE != 0)
        atomicAdd(&eacc[0], dE);
    if constexpr (SPLIT)
        if (dC != 0)
            atomicAdd(&eacc[1], dC);
    __syncthreads();
    if (tid == 0) {
        a.E[r] += eacc[0];
        if constexpr (SPLIT)
            a.C[r] += eacc[1];
    }
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        if (lv[c] < INT_MAX / 2) {
            const int p = tid + c * T;
            const int q = (RNG == 0) ? a.site[p] : site[p];
            int8_t* sp = a.spins + size_t(r) * N + q;
            FT* fg = static_cast<FT*>(a.fields) + size_t(r) * N + q;
            const int jt = jd[c] >> 8;
            for (int t = 0; t < M; ++t) {
                uint32_t w3;
                if constexpr (LONG) {
                    const int tm = t == 0 ? M - 1 : t - 1, tp = t + 1 == M ? 0 : t + 1;
                    w3 = ((colw[p * KW + (tm >> 5)] >> (tm & 31)) & 1u) |
                         (((colw[p * KW + (t >> 5)] >> (t & 31)) & 1u) << 1) |
                         (((colw[p * KW + (tp >> 5)] >> (tp & 31)) & 1u) << 2);
                } else {
                    w3 = __funnelshift_r(bits[c], bits[c], (t - 1) & 31);
                }
                sp[size_t(t) * S] = ((w3 >> 1) & 1u) ? int8_t(1) : int8_t(-1);
                fg[size_t(t) * S] =
                    FT(Fsp<FT>::ld(fsp, fb[c] + t) + jt * (2 * int((w3 & 1u) + ((w3 >> 2) & 1u)) - 2));
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

template <typename FT, int RNG, int CMAX, bool SMALL, bool LONG = false, bool SPLIT = false>
__global__ void __launch_bounds__(lean_bound_threads(CMAX, SMALL), lean_bound_blocks(CMAX, SMALL, RNG, SPLIT))
    lean_kernel(const SweepArgs a)
{
    lean_body<FT, RNG, CMAX, LONG, SPLIT>(a, int(blockIdx.x), int(gridDim.x));
}

// Batched launch over many instances: each block copies its instance's
// arguments into shared memory (so that every later read is a shared load).
template <typename FT, int RNG, int CMAX, bool SMALL, bool LONG = false>
__global__ void __launch_bounds__(lean_bound_threads(CMAX, SMALL), lean_bound_blocks(CMAX, SMALL, RNG))
    lean_batch_kernel(const SweepArgs* __restrict__ args, const BatchItem* __restrict__ items)
{
    __shared__ SweepArgs sa;
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0)
        sa = args[it.inst];
    __syncthreads();
    lean_body<FT, RNG, CMAX, LONG>(sa, it.block, sa.inst_blocks);
}

template <typename FT, int RNG>
void* pick_lean(int cmax, bool batch = false, bool small = false, bool longc = false)
{
    if (longc)  // M a multiple of 32 above 32: one or two columns per thread
        return cmax == 1 ? (batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 1, false, true>)
                                  : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 1, false, true>))
             : cmax == 2 ? (batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 2, false, true>)
                                  : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, false, true>))
                         : nullptr;
    if (small)  // two columns per thread only
        return cmax != 2 ? nullptr
                         : (batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 2, true>)
                                  : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, true>));
    switch (cmax) {
    case 1: return batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 1, false>)
                   : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 1, false>);
    case 2: return batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 2, false>)
                   : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, false>);
    case 4: return batch ? reinterpret_cast<void*>(&lean_batch_kernel<FT, RNG, 4, false>)
                   : reinterpret_cast<void*>(&lean_kernel<FT, RNG, 4, false>);
    default: return nullptr;
    }
}

// The split-coupling instantiations (single-instance launches only).
template <typename FT, int RNG>
void* pick_lean_split(int cmax, bool small, bool longc)
{
    if (longc)
        return cmax == 1 ? reinterpret_cast<void*>(&lean_kernel<FT, RNG, 1, false, true, true>)
             : cmax == 2 ? reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, false, true, true>)
                         : nullptr;
    if (small)
        return cmax == 2 ? reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, true, false, true>) : nullptr;
    switch (cmax) {
    case 1: return reinterpret_cast<void*>(&lean_kernel<FT, RNG, 1, false, false, true>);
    case 2: return reinterpret_cast<void*>(&lean_kernel<FT, RNG, 2, false, false, true>);
    case 4: return reinterpret_cast<void*>(&lean_kernel<FT, RNG, 4, false, false, true>);
    default: return nullptr;
    }
}

}  // namespace lean_detail

void* lean_kernel_i16(int rng, int cmax, bool batch = false, bool small = false, bool longc = false);
void* lean_kernel_i32(int rng, int cmax, bool batch = false, bool small = false, bool longc = false);
// split couplings (lean_split_i16.cu, lean_split_i32.cu)
void* lean_split_kernel_i16(int rng, int cmax, bool small, bool longc);
void* lean_split_kernel_i32(int rng, int cmax, bool small, bool longc);

}  // namespace isg
