// Track-scheduled wavefront sweep for the layered models of the paper's QMC
// setting (section 3.1): one replica per block, M in {4, 8, 16, 32} slices,
// spatial degree <= 6, |J| <= 63.  Same schedule, state and fused-PT protocol
// as the lean kernel (lean_impl.cuh): level(q, t) = lev0(q) + t, a barrier
// between levels, spatial fields in shared memory with atomic neighbour
// updates, column bits and random-word blocks in registers.
//
// What changes is who works on a level.  Column q is busy only during the M
// levels lev0(q) .. lev0(q) + M - 1 of the D levels of a sweep, so a thread
// that owns fixed columns idles most levels.  Here the columns are packed on
// the host into tracks: sequences of columns whose busy windows do not
// overlap (greedy in lev0 order; the number of tracks is the largest number
// of columns busy at one level).  Thread k walks track k: it carries one
// column in registers, stores its bits in shared memory when its window
// closes and loads the next column of the track.  A block therefore needs as
// many threads as the widest level, and almost every thread has an item on
// almost every level.
//
// Random words follow the thread's sequence of 4-word blocks across its
// columns: two blocks in flight, block j+1 fetched (MT19937, cp.async into the
// thread's own staging slot) or computed (Philox) when block j starts.
#pragma once
#include <climits>

#include "fast_impl.cuh"

namespace isg {
namespace track_detail {

using fast_detail::grid_sync;
using fast_detail::rng_block;

constexpr int kMaxDeg = 6;

struct TrackLayout {
    uint32_t colbits, stage, fsp, thr, eacc, slot, temp, total;
};

// Shared memory holds only what a level touches (spatial fields, thresholds)
// and the per-thread column state; the slice tables are read through the
// read-only cache when a thread opens a column (every M levels).
__host__ __device__ inline TrackLayout track_layout(const SweepArgs& a, int fbytes, int threads)
{
    TrackLayout L{};
    uint32_t o = 0;
    L.colbits = o; o += r16(4u * a.S);
    L.stage = o;   o += (a.rng == 0) ? r16(32u * uint32_t(threads)) : 0u;
    L.fsp = o;     o += r16(uint32_t(fbytes) * a.N);
    L.thr = o;     o += r16(4u * a.K);
    L.eacc = o;    o += 16u;
    if (a.swap_every > 0) {
        L.slot = o; o += r16(4u * a.R);
        L.temp = o; o += r16(4u * a.R);
    }
    L.total = o;
    return L;
}

// Body of one block: `blk` is the replica (block) index within its instance
// and `nblk` the instance's number of blocks.
template <typename FT, int RNG>
__device__ __forceinline__ void track_body(const SweepArgs& a, const int blk, const int nblk)
{
    constexpr bool kI16 = sizeof(FT) == 2;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    const int T = blockDim.x, tid = threadIdx.x;
    const TrackLayout L = track_layout(a, Fsp<FT>::kBytes, T);
    const int S = a.S, M = a.M, N = a.N, K = a.K, R = a.R;
    const int r = blk;
    const int* nbr_off = a.nbr_off;
    const uint32_t* nbr = a.nbr;
    const int* jtau = a.jtau;
    const int* pos = a.pos;
    const int* site = a.site;
    const int* lev0 = a.lev0;
    uint32_t* colbits = reinterpret_cast<uint32_t*>(smem + L.colbits);
    unsigned char* stage = smem + L.stage + tid * 32;  // MT19937: this thread's two 16-byte slots
    void* fsp = smem + L.fsp;
    unsigned* fsw = reinterpret_cast<unsigned*>(smem + L.fsp);
    uint32_t* thr_s = reinterpret_cast<uint32_t*>(smem + L.thr);
    int* eacc = reinterpret_cast<int*>(smem + L.eacc);
    int* slot_s = reinterpret_cast<int*>(smem + L.slot);
    int* temp_s = reinterpret_cast<int*>(smem + L.temp);
    const bool fused = a.swap_every > 0;

    // ---- labels, spatial fields, column bits, thresholds
    if (tid == 0)
        eacc[0] = 0;
    if (fused)
        for (int i = tid; i < R; i += T) {
            slot_s[i] = a.slot_of_temp[i];
            temp_s[i] = a.temp_of_slot[i];
        }
    __syncthreads();  // temp_s is read below
    const uint32_t rep = (M == 32) ? 1u : (M == 16 ? 0x00010001u : (M == 8 ? 0x01010101u : 0x11111111u));
    {
        const int8_t* sp = a.spins + size_t(r) * N;
        const FT* fg = static_cast<const FT*>(a.fields) + size_t(r) * N;
        for (int i = tid; i < N; i += T) {
            const int t = i / S, q = i - t * S, p = __ldg(pos + q);
            const int tm = (t == 0) ? M - 1 : t - 1, tp = (t == M - 1) ? 0 : t + 1;
            const int ft = __ldg(jtau + p) * (int(sp[tm * S + q]) + int(sp[tp * S + q]));
            Fsp<FT>::st(fsp, p * M + t, int(fg[i]) - ft);
        }
        for (int p = tid; p < S; p += T) {
            const int8_t* c = sp + __ldg(site + p);
            uint32_t b = 0u;
            for (int t = 0; t < M; ++t)
                b |= (c[size_t(t) * S] > 0 ? 1u : 0u) << t;
            colbits[p] = b * rep;  // the column replicated with period M
        }
    }
    {
        const int temp = fused ? temp_s[r] : a.temp_of_slot[r];
        for (int k = tid; k < K; k += T)
            thr_s[k] = a.thr[size_t(temp) * K + k];
    }
    __syncthreads();

    // ---- this thread's track: columns track_col[c0 .. c1) in time order
    const bool has = tid < a.ntracks;
    const int c0 = has ? __ldg(a.track_off + tid) : 0;
    const int c1 = has ? __ldg(a.track_off + tid + 1) : 0;
    const int nrb = (M + 3) >> 2;  // random-word blocks per column
    const unsigned FULL = 0xFFFFFFFFu;
    const bool shfl_thr = K <= 32;
    uint32_t thr_lane = (shfl_thr && (tid & 31) < K) ? thr_s[tid & 31] : 0u;
    const unsigned long long sweep0 = a.counters[0];
    const unsigned long long pass0 = a.counters[1];
    int npass = 0;
    int dE = 0;

    // current column (p, its site q, level window, Trotter coupling and
    // degree, field base, neighbour words, bits) and the next column's
    // metadata, loaded one column ahead so that no table read sits on a level
    int ci = c0, p = 0, q = 0, lev = INT_MAX / 2, jd = 0, fb = 0, jbase = 0;
    uint32_t bits = 0u;
    uint32_t nb[kMaxDeg];
    int np = 0, nq = 0, nlev = INT_MAX / 2, njd = 0;
    uint32_t nnb[kMaxDeg];
    uint4 ba = make_uint4(0u, 0u, 0u, 0u), bb = ba;  // Philox blocks of even / odd sequence index
    auto prefetch_meta = [&](int c) {
        np = __ldg(a.track_col + c);
        nq = __ldg(site + np);
        nlev = __ldg(lev0 + np);
        const int e0 = __ldg(nbr_off + np), deg = __ldg(nbr_off + np + 1) - e0;
        njd = (__ldg(jtau + np) << 8) | deg;
        const uint32_t own = kI16 ? uint32_t(np * M / 2) : uint32_t(np * M);
#pragma unroll
        for (int e = 0; e < kMaxDeg; ++e) {
            nnb[e] = own << 8;  // padding: zero delta on the own field word
            if (e < deg) {
                const uint32_t en = __ldg(nbr + e0 + e);
                const int q2 = int(en >> 16);
                const int twoJ = 2 * int(int16_t(en & 0xFFFFu));
                const uint32_t word = kI16 ? uint32_t(q2 * M / 2) : uint32_t(q2 * M);
                nnb[e] = (word << 8) | (uint32_t(twoJ) & 0xFFu);
            }
        }
    };
    auto take_next = [&]() {
        p = np;
        q = nq;
        lev = nlev;
        jd = njd;
        fb = p * M;
#pragma unroll
        for (int e = 0; e < kMaxDeg; ++e)
            nb[e] = nnb[e];
        bits = colbits[p];
    };
    // fetch block b of the column at position pp (site qq) into sequence slot s
    auto fetch = [&](int pp, int qq, int b, int s, const uint32_t* wsw, uint32_t sid) {
        if (RNG == 0) {
            cp_async16(stage + s * 16, wsw + (size_t(r) * S + pp) * a.Mp + 4 * b);
        } else {
            const uint4 v = rng_block<RNG>(a, wsw, r, pp, qq, b, sid);
            if (s)
                bb = v;
            else
                ba = v;
        }
    };
    if (c0 < c1)
        prefetch_meta(c0);

    for (int sw = 0; sw < a.nsweeps; ++sw) {
        const uint32_t sid = uint32_t(sweep0 + sw);
        const uint32_t* wsw = (RNG == 0) ? a.wbuf + size_t(sw) * a.wbuf_sweep_stride : nullptr;
        ci = c0;
        jbase = 0;
        lev = INT_MAX / 2;
        if (ci < c1) {
            take_next();
            prefetch_meta(ci + 1 < c1 ? ci + 1 : c0);
            fetch(p, q, 0, 0, wsw, sid);  // sequence blocks 0 and 1
            if (nrb > 1)
                fetch(p, q, 1, 1, wsw, sid);
            else if (ci + 1 < c1)
                fetch(np, nq, 0, 1, wsw, sid);
        }
        for (int l = 0; l < a.D; ++l) {
            if (ci < c1 && l == lev + M) {  // the column's window closed
                colbits[p] = bits;
                jbase += nrb;
                if (++ci < c1) {
                    take_next();
                    prefetch_meta(ci + 1 < c1 ? ci + 1 : c0);  // wraps to the next sweep's first column
                } else {
                    lev = INT_MAX / 2;
                }
            }
            const int t0 = l - lev;
            const bool act = ci < c1 && unsigned(t0) < unsigned(M);
            if (__any_sync(FULL, act)) {
                // converged section: every lane runs it, idle lanes on slice 0 of column 0
                const int t = act ? t0 : 0;
                const int j = jbase + (t >> 2);  // sequence index of the word block
                if (RNG == 0 && act && (t & 3) == 0)
                    cp_async_wait_all();  // block j has landed in its slot
                const int fs = Fsp<FT>::ld(fsp, act ? fb + t : 0);
                const uint32_t u = (RNG == 0)
                    ? *reinterpret_cast<const uint32_t*>(stage + (j & 1) * 16 + (t & 3) * 4)
                    : pick4((j & 1) ? bb : ba, t & 3);
                const uint32_t w3 = __funnelshift_r(bits, bits, (t - 1) & 31);
                const int s = 2 * int((w3 >> 1) & 1u) - 1;
                const int ft = (jd >> 8) * (2 * int((w3 & 1u) + ((w3 >> 2) & 1u)) - 2);
                const int k = s * (fs + ft);
                uint32_t tk;
                if (shfl_thr)
                    tk = __shfl_sync(FULL, thr_lane, (k > 0 && k < K) ? k : 0);
                else
                    tk = (k > 0 && k < K) ? thr_s[k] : 0u;
                if (act && ((k <= 0) || (k < K && u < tk))) {
                    bits ^= rep << t;
                    dE += 2 * k;
                    const int tw = kI16 ? (t >> 1) : t;
                    const int sh = kI16 ? ((t & 1) << 4) : 0;
#pragma unroll
                    for (int e = 0; e < kMaxDeg; ++e) {
                        const uint32_t v = nb[e];
                        const int d = -s * int(int8_t(v & 0xFFu));
                        atomicAdd(fsw + (v >> 8) + tw, unsigned(d) << sh);
                    }
                }
                // block j + 1 of the sequence replaces block j - 1 in the idle slot
                if (act && (t & 3) == 0 && j >= 1) {
                    if ((t >> 2) + 1 < nrb)
                        fetch(p, q, (t >> 2) + 1, (j + 1) & 1, wsw, sid);
                    else if (ci + 1 < c1)
                        fetch(np, nq, 0, (j + 1) & 1, wsw, sid);
                }
            }
            __syncthreads();
        }
        if (ci < c1)
            colbits[p] = bits;  // the track's last column

        if (fused && (sw + 1) % a.swap_every == 0) {
            if (dE != 0)
                atomicAdd(&eacc[0], dE);
            dE = 0;
            __syncthreads();
            int* Ep = a.E_pub + size_t(npass & 1) * R;
            if (tid == 0) {
                const int e = a.E[r] + eacc[0];
                a.E[r] = e;
                Ep[r] = e;
                eacc[0] = 0;
            }
            if (nblk == 1)  // a one-block instance has nobody else to wait for
                __syncthreads();
            else if (!grid_sync(a.gridbar, unsigned(npass + 1) * unsigned(nblk), a.err, &s_flag))
                return;
            if (tid < 32) {
                const unsigned long long pp = pass0 + npass;
                const int par = int(pp & 1ull);
                const int npairs = par ? (R - 1) / 2 : R / 2;
                for (int jj = tid; jj < npairs; jj += 32) {
                    const int kk = 2 * jj + par;
                    const int sa = slot_s[kk], sb = slot_s[kk + 1];
                    const long long d = (long long)__ldcg(Ep + sa) - (long long)__ldcg(Ep + sb);
                    uint32_t uu;
                    if (RNG == 0)
                        uu = a.swbuf[size_t(npass) * a.maxpairs + jj];
                    else
                        uu = pick4(philox4x32_10(make_uint4(uint32_t(jj) >> 2, uint32_t(pp), a.inst, 1u), a.seed,
                                                 0xFFFFFFFFu),
                                   jj & 3);
                    if ((d <= 0) || (d < a.swlen[kk] && uu < a.swthr[a.swoff[kk] + d])) {
                        slot_s[kk] = sb;
                        slot_s[kk + 1] = sa;
                        temp_s[sa] = kk + 1;
                        temp_s[sb] = kk;
                        if (blk == 0)
                            a.swap_acc[kk] += 1ull;
                    }
                }
            }
            __syncthreads();
            for (int kk = tid; kk < K; kk += T)
                thr_s[kk] = a.thr[size_t(temp_s[r]) * K + kk];
            __syncthreads();
            thr_lane = (shfl_thr && (tid & 31) < K) ? thr_s[tid & 31] : 0u;
            ++npass;
        }
    }

    // ---- energies and write-back of the track's columns
    if (dE != 0)
        atomicAdd(&eacc[0], dE);
    __syncthreads();
    if (tid == 0)
        a.E[r] += eacc[0];
    for (int c = c0; c < c1; ++c) {
        const int pp = __ldg(a.track_col + c);
        const uint32_t b = colbits[pp];
        const int q = __ldg(site + pp);
        int8_t* sp = a.spins + size_t(r) * N + q;
        FT* fg = static_cast<FT*>(a.fields) + size_t(r) * N + q;
        const int jt = __ldg(jtau + pp);
        for (int t = 0; t < M; ++t) {
            const uint32_t w3 = __funnelshift_r(b, b, (t - 1) & 31);
            sp[size_t(t) * S] = ((w3 >> 1) & 1u) ? int8_t(1) : int8_t(-1);
            fg[size_t(t) * S] = FT(Fsp<FT>::ld(fsp, pp * M + t) + jt * (2 * int((w3 & 1u) + ((w3 >> 2) & 1u)) - 2));
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

template <typename FT, int RNG>
__global__ void __launch_bounds__(512, 1) track_kernel(const SweepArgs a)
{
    track_body<FT, RNG>(a, int(blockIdx.x), int(gridDim.x));
}

// Batched launch over many instances (see lean_batch_kernel).
template <typename FT, int RNG>
__global__ void __launch_bounds__(512, 1)
    track_batch_kernel(const SweepArgs* __restrict__ args, const BatchItem* __restrict__ items)
{
    __shared__ SweepArgs sa;
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0)
        sa = args[it.inst];
    __syncthreads();
    track_body<FT, RNG>(sa, it.block, sa.inst_blocks);
}

template <typename FT, int RNG>
void* pick_track(bool batch)
{
    return batch ? reinterpret_cast<void*>(&track_batch_kernel<FT, RNG>)
                 : reinterpret_cast<void*>(&track_kernel<FT, RNG>);
}

}  // namespace track_detail

void* track_kernel_i16(int rng, bool batch = false);
void* track_kernel_i32(int rng, bool batch = false);

}  // namespace isg
