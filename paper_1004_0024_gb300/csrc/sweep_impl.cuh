// Wavefront Metropolis sweep (Figure 1 of Dickson, Karimi & Hamze, with the
// Figure 6 neighbour update) for M identical slices of S sites.
//
// Exactness.  Spin i's decision reads f_i after every neighbour j < i has
// been visited in the current sweep and before any neighbour j > i is.  The
// random word of each visit is fixed in advance (it does not depend on the
// decisions), so any schedule that visits i after all its lower-indexed
// neighbours and before all its higher-indexed neighbours reproduces the
// sequential sweep bit for bit.  With level(q, t) = lev0(q) + t, where lev0
// is the wavefront level of site q in the slice graph (1 + max over lower
// spatial neighbours), every edge (i, j), i < j, has level(i) < level(j):
// spatial edges by construction, Trotter edges because t grows by one, and
// the ring's wrap edge (q, 0)-(q, M-1) because M-1 >= 1.  So the block walks
// the levels in order with a barrier between levels; spins of one level are
// never adjacent and only ever add to shared fields with atomics.
//
// Work split.  A block holds G replicas; thread `tid` owns the columns
// x = tid + c*T (x = p*G + g, p = sorted site position, g = replica).  Column
// (p, g) is active at levels lev0(p) .. lev0(p)+M-1, one spin per level.  The
// column's spins are bits of colbits (touched only by the owner thread); the
// spatial part of every field lives in fsp and receives the neighbours'
// updates through shared-memory atomics; the Trotter part is recomputed from
// the owner's bits (the paper keeps h_eff_tau apart for the same reason).
#pragma once
#include <climits>

#include "field_ops.cuh"
#include "ising_internal.cuh"

namespace isg {
namespace sweep_detail {

struct SmemLayout {
    uint32_t nbr_off, nbr, jtau, pos, site, colbits, fsp, thr, eacc, stage, total;
};

__host__ __device__ inline SmemLayout smem_layout(const SweepArgs& a, int fbytes)
{
    SmemLayout L{};
    uint32_t o = 16;  // mbarrier
    if (a.tables_smem) {
        L.nbr_off = o; o += r16(4u * (a.S + 1));
        L.nbr = o;     o += r16(4u * (a.nbr_count > 0 ? a.nbr_count : 1));
        L.jtau = o;    o += r16(4u * a.S);
        L.pos = o;     o += r16(4u * a.S);
        L.site = o;    o += r16(4u * a.S);
    }
    L.colbits = o; o += r16(4u * a.S * a.G * a.W);
    L.fsp = o;     o += r16(uint32_t(fbytes) * a.N * a.G);
    if (a.thr_smem) { L.thr = o; o += r16(4u * a.G * a.K); }
    L.eacc = o;    o += r16(4u * a.G);
    if (a.stage_words) { L.stage = o; o += r16(32u * a.S * a.G); }  // [column x][2 blocks][4 words]
    L.total = o;
    return L;
}



template <typename FT, int RNG, int CMAX>
__global__ void __launch_bounds__(1024, 1) sweep_kernel(const SweepArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_fail;
    const SmemLayout L = smem_layout(a, Fsp<FT>::kBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    const int T = blockDim.x, tid = threadIdx.x;
    const int S = a.S, M = a.M, W = a.W, N = a.N, G = a.G, K = a.K;
    const int r0 = blockIdx.x * G;
    const int Gb = min(G, a.R - r0);

    const int* nbr_off = a.tables_smem ? reinterpret_cast<const int*>(smem + L.nbr_off) : a.nbr_off;
    const uint32_t* nbr = a.tables_smem ? reinterpret_cast<const uint32_t*>(smem + L.nbr) : a.nbr;
    const int* jtau = a.tables_smem ? reinterpret_cast<const int*>(smem + L.jtau) : a.jtau;
    const int* pos = a.tables_smem ? reinterpret_cast<const int*>(smem + L.pos) : a.pos;
    const int* site = a.tables_smem ? reinterpret_cast<const int*>(smem + L.site) : a.site;
    uint32_t* colbits = reinterpret_cast<uint32_t*>(smem + L.colbits);
    void* fsp = smem + L.fsp;
    uint32_t* thr_s = reinterpret_cast<uint32_t*>(smem + L.thr);
    int* eacc = reinterpret_cast<int*>(smem + L.eacc);

    // ---- stage the slice tables with bulk copies (one thread issues them)
    if (a.tables_smem && tid == 0)
        mbar_init(bar, 1);
    __syncthreads();
    if (a.tables_smem && tid == 0) {
        const uint32_t b0 = r16(4u * (S + 1)), b1 = r16(4u * (a.nbr_count > 0 ? a.nbr_count : 1));
        const uint32_t b2 = r16(4u * S);
        mbar_expect_tx(bar, b0 + b1 + 3 * b2);
        bulk_g2s(smem + L.nbr_off, a.nbr_off, b0, bar);
        bulk_g2s(smem + L.nbr, a.nbr, b1, bar);
        bulk_g2s(smem + L.jtau, a.jtau, b2, bar);
        bulk_g2s(smem + L.pos, a.pos, b2, bar);
        bulk_g2s(smem + L.site, a.site, b2, bar);
    }
    for (int i = tid; i < S * G * W; i += T)
        colbits[i] = 0u;
    for (int i = tid; i < G; i += T)
        eacc[i] = 0;
    if (tid == 0)
        s_fail = a.tables_smem ? !mbar_wait(bar, 0, kWaitPolls) : 0;
    __syncthreads();
    if (s_fail) {
        if (tid == 0)
            set_err(a.err, kErrTimeout);
        return;
    }
    if (a.tables_smem)
        mbar_wait(bar, 0, kWaitPolls);  // phase already complete: per-thread acquire

    // ---- replica state: spins -> column bits, total field -> spatial field
    for (int g = 0; g < Gb; ++g) {
        const int8_t* sp = a.spins + size_t(r0 + g) * N;
        for (int i = tid; i < N; i += T) {
            if (sp[i] > 0) {
                const int t = i / S, q = i - t * S;
                atomicOr(&colbits[(pos[q] * G + g) * W + (t >> 5)], 1u << (t & 31));
            }
        }
    }
    __syncthreads();
    for (int g = 0; g < Gb; ++g) {
        const FT* fg = static_cast<const FT*>(a.fields) + size_t(r0 + g) * N;
        for (int i = tid; i < N; i += T) {
            const int t = i / S, q = i - t * S, p = pos[q];
            const int ft = trotter_field(colbits + (p * G + g) * W, t, M, jtau[p]);
            Fsp<FT>::st(fsp, (p * M + t) * G + g, int(fg[i]) - ft);
        }
    }
    if (a.thr_smem) {
        for (int idx = tid; idx < Gb * K; idx += T) {
            const int g = idx / K, k = idx - g * K;
            thr_s[idx] = a.thr[size_t(a.temp_of_slot[r0 + g]) * K + k];
        }
    }
    __syncthreads();

    // ---- owned columns
    const int g = tid % G;
    const bool live = g < Gb;
    const int SG = S * G;
    int lv[CMAX];
#pragma unroll
    for (int c = 0; c < CMAX; ++c) {
        const int x = tid + c * T;
        lv[c] = (live && x < SG) ? a.lev0[x / G] : (INT_MAX / 2);
    }
    const uint32_t* thr_g =
        a.thr_smem ? thr_s + g * K : a.thr + size_t(live ? a.temp_of_slot[r0 + g] : 0) * K;
    const int rg = r0 + g;
    const unsigned long long sweep0 = a.counters[0];
    const int nrb = (M + 3) >> 2;  // 4-word blocks per column
    unsigned char* stage = smem + L.stage;
    int dE = 0;
    // words t = 4b .. 4b+3 of column x (position p) into staging slot b & 1
    auto fill = [&](const uint32_t* wsw, uint32_t sid, int x, int p, int b) {
        unsigned char* dst = stage + x * 32 + (b & 1) * 16;
        if (RNG == 0) {
            cp_async16(dst, wsw + (size_t(rg) * S + p) * a.Mp + 4 * b);
        } else {
            const uint4 ctr = make_uint4(uint32_t(b * S + site[p]), sid, a.inst, 0u);
            *reinterpret_cast<uint4*>(dst) = philox4x32_10(ctr, a.seed, uint32_t(rg));
        }
    };

    for (int sw = 0; sw < a.nsweeps; ++sw) {
        const uint32_t sid = uint32_t(sweep0 + sw);
        const uint32_t* wsw = (RNG == 0) ? a.wbuf + size_t(sw) * a.wbuf_sweep_stride : nullptr;
        if (a.stage_words) {  // blocks 0 and 1 of every owned column
#pragma unroll
            for (int c = 0; c < CMAX; ++c) {
                const int x = tid + c * T;
                if (lv[c] < INT_MAX / 2) {
                    fill(wsw, sid, x, x / G, 0);
                    if (nrb > 1)
                        fill(wsw, sid, x, x / G, 1);
                }
            }
        }
        for (int l = 0; l < a.D; ++l) {
#pragma unroll
            for (int c = 0; c < CMAX; ++c) {
                const int t = l - lv[c];
                if (unsigned(t) < unsigned(M)) {
                    const int p = (tid + c * T) / G;
                    uint32_t* cb = colbits + (p * G + g) * W;
                    const uint32_t cw = cb[t >> 5];
                    const int up = (cw >> (t & 31)) & 1;
                    const int fidx = (p * M + t) * G + g;
                    const int f = Fsp<FT>::ld(fsp, fidx) + trotter_field(cb, t, M, jtau[p]);
                    const int s = 2 * up - 1;
                    const int k = s * f;
                    uint32_t u;
                    if (a.stage_words) {
                        const int x = tid + c * T;
                        if (RNG == 0 && (t & 3) == 0)
                            cp_async_wait_all();  // block t>>2 has landed
                        u = reinterpret_cast<const uint32_t*>(stage + x * 32 + ((t >> 2) & 1) * 16)[t & 3];
                        // block (t>>2)+1 replaces block (t>>2)-1 in the idle slot
                        if ((t & 3) == 0 && t > 0 && (t >> 2) + 1 < nrb)
                            fill(wsw, sid, x, p, (t >> 2) + 1);
                    } else if (RNG == 0) {
                        u = wsw[(size_t(rg) * S + p) * a.Mp + t];
                    } else {
                        const uint4 ctr = make_uint4(uint32_t((t >> 2) * S + site[p]), sid, a.inst, 0u);
                        u = pick4(philox4x32_10(ctr, a.seed, uint32_t(rg)), t & 3);
                    }
                    const bool acc = (k <= 0) || (k < K && u < thr_g[k]);
                    if (acc) {
                        cb[t >> 5] = cw ^ (1u << (t & 31));
                        dE += 2 * k;
                        const int m2s = -2 * s;
                        const int e1 = nbr_off[p + 1];
                        for (int e = nbr_off[p]; e < e1; ++e) {
                            const uint32_t en = nbr[e];
                            const int q2 = int(en >> 16);
                            const int J = int(int16_t(en & 0xFFFFu));
                            Fsp<FT>::add(fsp, (q2 * M + t) * G + g, m2s * J);
                        }
                    }
                }
            }
            __syncthreads();
        }
    }

    // ---- energies and write-back
    if (live && dE != 0)
        atomicAdd(&eacc[g], dE);
    __syncthreads();
    if (tid < Gb)
        a.E[r0 + tid] += eacc[tid];
    for (int gg = 0; gg < Gb; ++gg) {
        int8_t* sp = a.spins + size_t(r0 + gg) * N;
        FT* fg = static_cast<FT*>(a.fields) + size_t(r0 + gg) * N;
        for (int i = tid; i < N; i += T) {
            const int t = i / S, q = i - t * S, p = pos[q];
            const uint32_t* cb = colbits + (p * G + gg) * W;
            const int up = (cb[t >> 5] >> (t & 31)) & 1;
            sp[i] = up ? int8_t(1) : int8_t(-1);
            fg[i] = FT(Fsp<FT>::ld(fsp, (p * M + t) * G + gg) + trotter_field(cb, t, M, jtau[p]));
        }
    }
    // the last block to finish advances the sweep counter
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(a.done_blocks, 1u);
        if (prev == gridDim.x - 1) {
            a.counters[0] += (unsigned long long)a.nsweeps;
            *a.done_blocks = 0u;
            __threadfence();
        }
    }
}

template <typename FT, int RNG>
void* pick_cmax(int cmax)
{
    switch (cmax) {
    case 1: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 1>);
    case 2: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 2>);
    case 4: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 4>);
    case 8: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 8>);
    case 16: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 16>);
    case 32: return reinterpret_cast<void*>(&sweep_kernel<FT, RNG, 32>);
    default: return nullptr;
    }
}

}  // namespace sweep_detail

// one translation unit per field width instantiates the kernels
void* sweep_kernel_i16(int rng, int cmax);
void* sweep_kernel_i32(int rng, int cmax);

}  // namespace isg
