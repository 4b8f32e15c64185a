// Packed (slot-scheduled) wavefront sweep: one replica per block of one or a
// few warps, the columns' busy windows packed by the host into thread slots.
//
// Schedule and exactness are those of the lean kernel (lean_impl.cuh): spin
// (q, t) runs at level lev0(q) + t, a block barrier separates levels, and
// the random words are fixed in advance, so any such order gives the chain
// of the sequential sweep of Figure 1 bit for bit.  What changes is who does
// the work of a level.  A column of M slices is busy during M consecutive
// levels [lev0, lev0 + M); the host packs the columns, in order of lev0, into
// "slots", each column into the lowest-numbered slot that is free at its
// start, a slot's next column starting no earlier than the first level
// divisible by 4 after the previous one's window (165 slots cover the 1024
// columns of the 32 x 32 lattice; its widest level has 152 busy columns).
// Thread `tid` of a block of T threads runs slots tid, tid + T, ... (RMAX of
// them, unrolled as "rounds").
//
// Per level a thread only does the items of its busy slots: six neighbour
// words, the random word, the decision, and on a flip one store of the
// column word (the level loop is unrolled by four).  Everything else happens
// every fourth level, at the same level for every thread (no divergence): at
// a level l divisible by 4, before its items, a slot whose next column starts
// in [l, l + 4) takes it up (one 64-byte descriptor from shared memory) and
// the word block fetched four levels earlier goes into the ring; after the
// items, the slot fetches its next word block.  The column words are placed
// in banks by the host so that a level's neighbour loads spread over them.
//
// Fields by gathering.  A visit computes the spatial field from the
// neighbours' column bits, f_space = (h_q - sum_j J_qj) + sum_j 2 J_qj b_j(t),
// with plain shared-memory loads of their column words, instead of keeping
// every field and pushing the changes of a flip into the neighbours' fields:
// on sm_103a a shared-memory reduction instruction costs about 40 cycles of
// a warp's time (measured), six of them per visit, while six plain loads
// issue back to back.  The values are the same by definition (f = h + sum J
// s), so the chain is unchanged; the fields handed back through the ABI are
// recomputed from the spins when the launch ends.  Shared memory then holds
// only the column words of the replica (bit t of column q = spin (q, t) is
// +1): the owner of a busy column keeps it in a register and stores it when
// a spin flips; a neighbour reading the word at the same level reads a slice
// other than the one being flipped (neighbours lie at different levels), so
// it sees the value of the sequential sweep: updated for a lower-indexed
// neighbour (visited at an earlier level), not yet for a higher-indexed one.
// The Trotter part of the field, Jtau (s_{t-1} + s_{t+1}), comes from the
// owner's register bits: the bits of a slice mask rotated by one each level
// and by one either way for the ring neighbours.
//
// Random words go through a ring of 16 levels per slot in shared memory: the
// word of the slot's item at level l sits at (l mod 16) NSP + sl, so a
// level's reads are conflict-free and their address is the same offset for
// every slot.  Words come from the word buffer: at a level l divisible by 4
// a slot loads the 4-word block that starts in levels [l + 8, l + 12) with
// one 16-byte load into registers and stores it into the ring at level l + 4
// (four plain stores to four ring levels; 4-byte asynchronous copies of
// scattered blocks cost several shared-memory wavefronts each); the ring
// then holds levels l .. l + 14.  The blocks of a sweep's first 8 levels are
// asynchronous copies requested before the sweep (during the PT pass).
// Without the generator warps, Philox blocks are computed by the slot, the
// ten rounds spread over four levels (3, 3, 3, 1), and stored after the
// fourth.  An entry is written after the last item that reads it.
//
// The words are generated inside the kernel: after its T sweep threads a
// block has `gen` more warps (two), which write the next sweep's words into a
// two-sweep buffer in global memory (in L2 for a resident ladder).  MT19937:
// they advance the replica's stream (its ring of 1024 words in shared memory;
// 227 consecutive words of the stream depend only on earlier ones and are
// computed in parallel), four slices at a time (two where shared memory is
// short) staged in shared memory and then one 16-byte (8-byte) store per
// column.  Philox: one call per column and 4-slice block.  The sweep threads synchronise levels with a
// barrier of their own; block-wide barriers at the start and end of a sweep
// hand a buffer half from the generator to the sweep threads and back.
//
// Fused PT: as in the lean kernel (publish the energies, bounded grid
// barrier, every block runs the same PT pass on its own copy of the labels).
#pragma once
#include <climits>
#include <type_traits>

#include "fast_impl.cuh"

namespace isg {
namespace packed_detail {

using fast_detail::grid_sync;

constexpr int kMaxDeg = 6;
constexpr int kGenWarps = 2;  // MT19937 generator warps per block
// descriptor words of the column at position p: [0] lev0 | site << 16,
// [1] byte offset of its column word (the host places the words so that the
// neighbour loads of a warp spread over the banks), [2] 2 Jtau, [3] the field constant
// h_q - sum_j J_qj - 2 Jtau, [4..9] byte offsets of the spatial neighbours'
// column words, [10..15] their 2 J (missing neighbours: the column itself
// with J = 0).  The kernel turns the byte offsets into shared-memory
// addresses once per launch.
constexpr int kDescWords = 16;

struct PackedLayout {
    uint32_t bar, desc, pos, soff, scol, colw, stage, thr, eacc, slot, temp, gring, gstg, total;
};

// Shared-memory layout; the table part (desc .. scol) is one bulk copy of the
// handle's packed table buffer, whose parts are padded identically.
__host__ __device__ inline PackedLayout packed_layout(const SweepArgs& a, int threads)
{
    PackedLayout L{};
    uint32_t o = 0;
    L.bar = o;   o += 16;
    L.desc = o;  o += 4u * kDescWords * uint32_t(a.S);
    L.pos = o;   o += r16(4u * uint32_t(a.S));
    L.soff = o;  o += r16(4u * uint32_t(a.nslots + 1));
    L.scol = o;  o += r16(4u * uint32_t(a.S));
    L.colw = o;  o += r16(4u * uint32_t(a.S) * uint32_t(a.M > 32 ? a.M / 32 : 1));  // M / 32 words per long column
    L.stage = o;  // the word ring: 16 levels x slots rounded up to whole rounds
    o += 64u * uint32_t((a.nslots + threads - 1) / threads) * uint32_t(threads);
    L.thr = o;   o += r16(4u * uint32_t(a.K));
    L.eacc = o;  o += 16;
    if (a.swap_every > 0) {
        L.slot = o; o += r16(4u * uint32_t(a.R));
        L.temp = o; o += r16(4u * uint32_t(a.R));
    }
    if (a.gen && a.rng == 0) {  // the MT19937 generator's stream ring and four staged slices
        L.gring = o; o += 4u * kMtRing;
        L.gstg = o;  o += 4u * (a.gen_slices == 2 ? 2u : 4u) * uint32_t(a.S);
    }
    L.total = o;
    return L;
}

// bytes of the table part (desc, pos, slot offsets, slot columns)
__host__ __device__ inline uint32_t packed_table_bytes(int S, int nslots)
{
    return 4u * kDescWords * uint32_t(S) + r16(4u * uint32_t(S)) + r16(4u * uint32_t(nslots + 1)) +
           r16(4u * uint32_t(S));
}

// 16-byte asynchronous copy without its own commit group.
__device__ __forceinline__ void cp_async16_nc(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void philox_round(uint4& c, uint32_t& k0, uint32_t& k1)
{
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
}

// LONG: columns of M = 32 W slices (W >= 2), stored word-major (word w of
// the column at slot c is colw[w S + c], so a warp's loads of different
// columns spread over the banks); a slot keeps the busy word and its two
// neighbours in registers.
template <int RNG, int RMAX, bool LONG = false>
__device__ __forceinline__ void packed_body(const SweepArgs& a, const int blk, const int nblk)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_flag;
    // T sweep threads (threads 0 .. T-1), then with the MT19937 generator
    // a.gen more warps (glane numbers their threads)
    const int T = a.sweep_threads, NT = blockDim.x, tid = threadIdx.x;
    // the generator warps make the words of both generators (Philox: one call
    // per column and 4-slice block); without them Philox words are made by
    // the slots themselves
    const bool gen = a.gen != 0;
    const bool ring_words = RNG == 0 || gen;  // words come from the word buffer
    const bool is_gen = gen && tid >= T;
    const int st = tid;
    const int glane = tid - T, GL = NT - T;  // generator threads
    const PackedLayout L = packed_layout(a, T);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    const int S = a.S, M = a.M, N = a.N, K = a.K, R = a.R;
    const int r = blk;  // one replica per block
    uint32_t* desc = reinterpret_cast<uint32_t*>(smem + L.desc);
    const int* pos = reinterpret_cast<const int*>(smem + L.pos);
    const int* soff = reinterpret_cast<const int*>(smem + L.soff);
    const int* scol = reinterpret_cast<const int*>(smem + L.scol);
    uint32_t* colw = reinterpret_cast<uint32_t*>(smem + L.colw);
    uint32_t* stage = reinterpret_cast<uint32_t*>(smem + L.stage);
    uint32_t* thr_s = reinterpret_cast<uint32_t*>(smem + L.thr);
    int* eacc = reinterpret_cast<int*>(smem + L.eacc);
    int* slot_s = reinterpret_cast<int*>(smem + L.slot);
    int* temp_s = reinterpret_cast<int*>(smem + L.temp);
    const bool fused = a.swap_every > 0;
    const bool f16 = a.field_bits == 16;

    // ---- tables (one bulk copy), labels
    if (tid == 0)
        mbar_init(bar, 1);
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(bar, a.pk_bytes);
        bulk_g2s(smem + L.desc, a.pk, a.pk_bytes, bar);
        eacc[0] = 0;
    }
    if (fused)
        for (int i = tid; i < R; i += NT) {
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

    // ---- column bits from the spins (the fields follow from them); the
    // descriptors' byte offsets become shared-memory addresses
    const uint32_t colw_s = smem_u32(colw), stage_s = smem_u32(stage);
    const int8_t* spg = a.spins + size_t(r) * N;
    for (int p = tid; p < S; p += NT) {
        uint32_t* d = desc + p * kDescWords;
        d[1] += colw_s;
#pragma unroll
        for (int e = 0; e < kMaxDeg; ++e)
            d[4 + e] += colw_s;
        const int q = int(d[0] >> 16);
        if constexpr (LONG) {
            for (int w = 0; w < M / 32; ++w) {
                uint32_t b = 0u;
                for (int t = 0; t < 32; ++t)
                    b |= (spg[size_t(32 * w + t) * S + q] > 0 ? 1u : 0u) << t;
                colw[((d[1] - colw_s) >> 2) + w * S] = b;
            }
        } else {
            uint32_t b = 0u;
            for (int t = 0; t < M; ++t)
                b |= (spg[size_t(t) * S + q] > 0 ? 1u : 0u) << t;
            colw[(d[1] - colw_s) >> 2] = b;
        }
    }
    {
        const int temp = fused ? temp_s[r] : a.temp_of_slot[r];
        for (int k = tid; k < K; k += NT)
            thr_s[k] = a.thr[size_t(temp) * K + k];
    }
    __syncthreads();

    const uint32_t rep = (LONG || M == 32) ? 1u : (M == 16 ? 0x00010001u : 0x01010101u);
    const uint32_t cmask = (LONG || M == 32) ? 0xFFFFFFFFu : ((1u << M) - 1u);
    const int nrb = M >> 2;  // word blocks per column
    const unsigned FULL = 0xFFFFFFFFu;
    const bool shfl_thr = K <= 32;
    uint32_t thr_lane = (shfl_thr && (tid & 31) < K) ? thr_s[tid & 31] : 0u;
    const unsigned long long sweep0 = a.counters[0];
    const unsigned long long pass0 = a.counters[1];
    const int NSP = ((a.nslots + T - 1) / T) * T;  // slots rounded up to whole rounds
    const uint32_t sbase = stage_s + 4u * uint32_t(st);  // the slot's ring column (round 0)
    const uint32_t lstride = 4u * uint32_t(NSP);          // bytes per ring level
    // ring column of each round; rounds past the last slot (always idle)
    // read round 0's
    uint32_t sbc[RMAX];
#pragma unroll
    for (int c = 0; c < RMAX; ++c)
        sbc[c] = sbase + (c * T < NSP ? 4u * uint32_t(c * T) : 0u);
    constexpr int kNone = INT_MAX / 2;
    int npass = 0;
    int dk = 0;  // sum of s_t f over the flips: the energy change is 2 dk

    // per slot (round c): the current column (busy, or the next to become
    // busy) and its successor in the slot's list
    int lv[RMAX] = {}, kk[RMAX] = {}, ke[RMAX] = {}, pp[RMAX] = {}, qq[RMAX] = {}, jt2[RMAX] = {};
    int pn[RMAX] = {}, qn[RMAX] = {}, ln[RMAX] = {};
    int cq[RMAX];       // h_q - sum_j J_qj - 2 Jtau
    uint32_t sa[RMAX];  // shared address of the column's own word
    // slice mask of the level: bit t of the column (t = level - lev0, with
    // the word's copies for M < 32), rotated by one each level
    uint32_t mrot[RMAX] = {};
    uint32_t bits[RMAX], nw[RMAX][kMaxDeg];  // nw: shared address of each neighbour's column word
    // LONG: the words before and after the busy one (for the Trotter bits at
    // a word's edges) and the address of the column's first word
    uint32_t wprev[RMAX] = {}, wnext[RMAX] = {}, sa0[RMAX] = {};
    int nj[RMAX][kMaxDeg];                    // 2 J of each neighbour
    // request cursor: the slot's next block to fetch (block xb of the column
    // at position xcol, site xsite, xk in the slot's list), its first level xx
    int xx[RMAX], xb[RMAX] = {}, xcol[RMAX] = {}, xsite[RMAX] = {}, xk[RMAX] = {};
    // block fetched at the last level divisible by 4 (16-byte load into
    // registers), stored into the ring at the next one; wx = its first level
    uint4 wq[RMAX];
    int wx[RMAX];
    // Philox block in progress: counter, keys, first level, whether any
    uint4 pc[RMAX] = {};
    uint32_t pk0[RMAX], pk1[RMAX];
    int px[RMAX];
    bool pgo[RMAX];

    // take up column p at level l (before the first of its items)
    auto load_col = [&](int c, int p, int l) {
        const uint4* d = reinterpret_cast<const uint4*>(desc + p * kDescWords);
        const uint4 d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3];
        lv[c] = int(d0.x & 0xFFFFu);
        qq[c] = int(d0.x >> 16);
        sa[c] = d0.y;
        jt2[c] = int(d0.z);
        cq[c] = int(d0.w);
        nw[c][0] = d1.x; nw[c][1] = d1.y; nw[c][2] = d1.z; nw[c][3] = d1.w; nw[c][4] = d2.x; nw[c][5] = d2.y;
        nj[c][0] = int(d2.z); nj[c][1] = int(d2.w); nj[c][2] = int(d3.x);
        nj[c][3] = int(d3.y); nj[c][4] = int(d3.z); nj[c][5] = int(d3.w);
        pp[c] = p;
        if constexpr (LONG) {
            const int w0 = int((d0.y - colw_s) >> 2), W = M / 32;
            sa0[c] = d0.y;
            bits[c] = colw[w0];
            wprev[c] = colw[w0 + (W - 1) * S];  // slice M - 1, the ring neighbour of slice 0
            wnext[c] = colw[w0 + S];
        } else {
            bits[c] = colw[(d0.y - colw_s) >> 2] * rep;
        }
        mrot[c] = __funnelshift_r(rep, rep, uint32_t(lv[c] - l));
    };
    auto set_next = [&](int c) {
        pn[c] = kk[c] + 1 < ke[c] ? scol[kk[c] + 1] : -1;
        const uint32_t d0 = pn[c] >= 0 ? desc[pn[c] * kDescWords] : 0u;
        qn[c] = int(d0 >> 16);
        ln[c] = pn[c] >= 0 ? int(d0 & 0xFFFFu) : kNone;
    };
    // slots restart at their first column (every column word is current:
    // owners store theirs at each flip; after a sweep's last level barrier
    // every thread sees them)
    auto restart = [&]() {
#pragma unroll
        for (int c = 0; c < RMAX; ++c) {
            const int sl = st + c * T;
            lv[c] = kNone;
            kk[c] = ke[c] = 0;
            pp[c] = qq[c] = jt2[c] = 0;
            pn[c] = -1;
            qn[c] = 0;
            ln[c] = kNone;
            cq[c] = 0;
            sa[c] = colw_s;
            bits[c] = 0u;
#pragma unroll
            for (int e = 0; e < kMaxDeg; ++e) {
                nw[c][e] = colw_s;
                nj[c][e] = 0;
            }
            pgo[c] = false;
            px[c] = 0;
            xx[c] = kNone;
            xb[c] = xcol[c] = xsite[c] = xk[c] = 0;
            wx[c] = kNone;
            wq[c] = make_uint4(0u, 0u, 0u, 0u);
            if (sl < a.nslots) {
                kk[c] = soff[sl];
                ke[c] = soff[sl + 1];
                if (kk[c] < ke[c]) {
                    load_col(c, scol[kk[c]], 0);
                    set_next(c);
                    xx[c] = lv[c];
                    xcol[c] = pp[c];
                    xsite[c] = qq[c];
                    xk[c] = kk[c];
                }
            }
        }
    };
    // Round c's next block if it starts in levels [l + 8, l + 12) (blocks are
    // fetched in order, one at most per window: a column's blocks start 4
    // levels apart and the slot's next column at least 4 after its last one),
    // and the cursor moved past it.
    auto next_block = [&](int c, int l, int& col, int& b, int& x, int& site) -> bool {
        if (xx[c] >= l + 12)
            return false;
        col = xcol[c];
        b = xb[c];
        x = xx[c];
        site = xsite[c];
        if (++xb[c] < nrb) {
            xx[c] += 4;
        } else if (++xk[c] < ke[c]) {
            xcol[c] = scol[xk[c]];
            const uint32_t d0 = desc[xcol[c] * kDescWords];
            xx[c] = int(d0 & 0xFFFFu);
            xsite[c] = int(d0 >> 16);
            xb[c] = 0;
        } else {
            xx[c] = kNone;
        }
        return true;
    };
    // ring address of round c's word for level x
    auto ring_addr = [&](int c, int x) {
        return sbase + 4u * uint32_t(c * T) + uint32_t(x & 15) * lstride;
    };
    // the block fetched four levels ago into its ring levels
    auto store_fetched = [&](int c) {
        if (wx[c] < kNone) {
            const uint32_t v[4] = {wq[c].x, wq[c].y, wq[c].z, wq[c].w};
#pragma unroll
            for (int w = 0; w < 4; ++w)
                asm volatile("st.shared.u32 [%0], %1;" ::"r"(ring_addr(c, wx[c] + w)), "r"(v[w]) : "memory");
            wx[c] = kNone;
        }
    };
    // in a sweep: the next block of every round, one 16-byte load into
    // registers (through L2: the generator warps write the buffer)
    auto fetch_words = [&](const uint32_t* wsw, int l) {
#pragma unroll
        for (int c = 0; c < RMAX; ++c) {
            int col = 0, b = 0, x = 0, site = 0;
            if (next_block(c, l, col, b, x, site)) {
                wq[c] = __ldcg(reinterpret_cast<const uint4*>(wsw + (size_t(r) * S + col) * a.Mp + 4 * b));
                wx[c] = x;
            }
        }
    };
    // at a sweep's start: 4-byte copies of the next block of every round into
    // its ring levels
    auto request_words = [&](const uint32_t* wsw, int l) {
#pragma unroll
        for (int c = 0; c < RMAX; ++c) {
            int col = 0, b = 0, x = 0, site = 0;
            if (next_block(c, l, col, b, x, site)) {
                const uint32_t* src = wsw + (size_t(r) * S + col) * a.Mp + 4 * b;
#pragma unroll
                for (int w = 0; w < 4; ++w)
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(ring_addr(c, x + w)),
                                 "l"(src + w)
                                 : "memory");
            }
        }
    };
    auto philox_store = [&](int c) {
        const uint32_t v[4] = {pc[c].x, pc[c].y, pc[c].z, pc[c].w};
#pragma unroll
        for (int w = 0; w < 4; ++w)
            asm volatile("st.shared.u32 [%0], %1;" ::"r"(ring_addr(c, px[c] + w)), "r"(v[w]) : "memory");
        pgo[c] = false;
    };
    // Philox: start (and with `full`, finish and store) the next blocks
    auto philox_start = [&](uint32_t sid, int l, bool full) {
#pragma unroll
        for (int c = 0; c < RMAX; ++c) {
            int col = 0, b = 0, x = 0, site = 0;
            pgo[c] = next_block(c, l, col, b, x, site);
            if (pgo[c]) {
                pc[c] = make_uint4(uint32_t(b * S + site), sid, a.inst, 0u);
                pk0[c] = a.seed;
                pk1[c] = uint32_t(r);
                px[c] = x;
                for (int i = 0; i < (full ? 10 : 3); ++i)
                    philox_round(pc[c], pk0[c], pk1[c]);
                if (full)
                    philox_store(c);
            }
        }
    };

    // ---- MT19937 generator warp
    uint32_t* gring = reinterpret_cast<uint32_t*>(smem + L.gring);
    uint32_t* gstg = reinterpret_cast<uint32_t*>(smem + L.gstg);
    uint32_t gw = 0u;  // low word of the stream position (ring slots need only these bits)
    // barrier of the generator warps (named barrier 2)
    auto gen_sync = [&]() { asm volatile("bar.sync 2, %0;" ::"r"(GL) : "memory"); };
    auto gen_sweep = [&](uint32_t* wdst) {
        const int lane = glane;
        const int G = a.gen_slices == 2 ? 2 : 4;  // slices staged per column store
        for (int t0 = 0; t0 < M; t0 += G) {
            const int group = G * S;
            for (int base = 0; base < group; base += kMtStep) {
                const int cnt = min(kMtStep, group - base);
                // the thread's (up to) 4 words of the step: their inputs first (all
                // of them from earlier steps), then the recurrences, then the stores
                constexpr int kPer = (kMtStep + 32 * kGenWarps - 1) / (32 * kGenWarps);
                uint32_t xa[kPer], xb[kPer], xm[kPer];
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const uint32_t w = gw + uint32_t(base + lane + GL * i);
                    xa[i] = gring[(w - 624u) & (kMtRing - 1)];
                    xb[i] = gring[(w - 623u) & (kMtRing - 1)];
                    xm[i] = gring[(w - 227u) & (kMtRing - 1)];
                }
#pragma unroll
                for (int i = 0; i < kPer; ++i) {
                    const int j = lane + GL * i;
                    if (j < cnt) {
                        const uint32_t w = gw + uint32_t(base + j);
                        const uint32_t x = mt_recur(xa[i], xb[i], xm[i]);
                        gring[w & (kMtRing - 1)] = x;
                        gstg[base + j] = mt_temper(x);
                    }
                }
                gen_sync();
            }
            // column q gets the words of slices t0 .. t0 + G - 1 as one 16-byte
            // (or 8-byte) store
            if (G == 4) {
                for (int q = lane; q < S; q += GL)
                    *reinterpret_cast<uint4*>(wdst + (size_t(r) * S + pos[q]) * a.Mp + t0) =
                        make_uint4(gstg[q], gstg[S + q], gstg[2 * S + q], gstg[3 * S + q]);
            } else {
                for (int q = lane; q < S; q += GL)
                    *reinterpret_cast<uint2*>(wdst + (size_t(r) * S + pos[q]) * a.Mp + t0) =
                        make_uint2(gstg[q], gstg[S + q]);
            }
            gen_sync();
            gw += uint32_t(group);
        }
    };
    // Philox: the blocks of every column for sweep id `sid`, 16 bytes each
    auto gen_sweep_philox = [&](uint32_t* wdst, uint32_t sid) {
        for (int p = glane; p < S; p += GL) {
            const int q = int(desc[p * kDescWords] >> 16);
            uint4* dst = reinterpret_cast<uint4*>(wdst + (size_t(r) * S + p) * a.Mp);
            for (int b = 0; b < nrb; ++b)
                dst[b] = philox4x32_10(make_uint4(uint32_t(b * S + q), sid, a.inst, 0u), a.seed, uint32_t(r));
        }
    };
    // the half of the two-sweep buffer for sweep sw (the handle's own word buffer)
    auto gen_buf = [&](int sw) { return const_cast<uint32_t*>(a.wbuf) + size_t(sw & 1) * a.wbuf_sweep_stride; };
    if (is_gen) {
        if (RNG == 0) {
            for (int i = glane; i < kMtRing; i += GL)
                gring[i] = a.mtring[size_t(r) * kMtRing + i];
            gw = uint32_t(a.mtpos[r]);
            gen_sync();
            if (a.nsweeps > 0)
                gen_sweep(gen_buf(0));
        } else if (a.nsweeps > 0) {
            gen_sweep_philox(gen_buf(0), uint32_t(sweep0));
        }
    }

    if (!is_gen)
        restart();
    __syncthreads();  // the first sweep's words are ready
    for (int sw = 0; sw < a.nsweeps; ++sw) {
        const uint32_t sid = uint32_t(sweep0 + sw);
        const uint32_t* wsw = gen ? gen_buf(sw) : (RNG == 0 ? a.wbuf + size_t(sw) * a.wbuf_sweep_stride : nullptr);
        if (is_gen) {
            // the generator: the next sweep's words while this one runs, handed over
            // at the sweep's end barrier
            __syncthreads();
            if (sw + 1 < a.nsweeps) {
                if (RNG == 0)
                    gen_sweep(gen_buf(sw + 1));
                else
                    gen_sweep_philox(gen_buf(sw + 1), uint32_t(sweep0 + sw + 1));
            }
            __syncthreads();
        } else {
        // the blocks that start in levels [0, 8)
        if (ring_words) {
            if (sw == 0) {  // later sweeps: requested at the end of the previous one
                request_words(wsw, -8);
                request_words(wsw, -4);
            }
            cp_async_commit();
            asm volatile("cp.async.wait_all;" ::: "memory");
        } else {
            philox_start(sid, -8, true);
            philox_start(sid, -4, true);
        }
        __syncthreads();  // sweep start (block-wide)

        // One level: the items first (the rounds are independent: a neighbour
        // of a busy spin is at another level, so all loads go first, then the
        // fields and decisions, then the stores of the flipped columns), then
        // the word stream, then the level barrier.  PH = l mod 4.
        auto level = [&](const int l, auto ph_c) {
            constexpr int PH = decltype(ph_c)::value;
            if (PH == 0) {
                if (ring_words) {
#pragma unroll
                    for (int c = 0; c < RMAX; ++c)
                        store_fetched(c);
                }
                // a slot takes up its next column at the last multiple of 4 before
                // the column's start (the previous one has ended by then: the host
                // packs a slot's next column at or after the first multiple of 4
                // past the previous window)
#pragma unroll
                for (int c = 0; c < RMAX; ++c) {
                    if (pn[c] >= 0 && (ln[c] & ~3) <= l) {
                        ++kk[c];
                        load_col(c, pn[c], l);
                        set_next(c);
                    }
                }
            }
            const uint32_t lofs = uint32_t(l & 15) * lstride;
            uint32_t mnext[RMAX];  // the next level's slice masks
#pragma unroll
            for (int c = 0; c < RMAX; ++c)
                mnext[c] = __funnelshift_l(mrot[c], mrot[c], 1);
            bool any = true;
            if (RMAX == 1)  // one round: a warp without a busy slot skips the level's items
                any = __any_sync(FULL, unsigned(l - lv[0]) < unsigned(M));
            if (any) {
                uint32_t uu[RMAX], wn[RMAX][kMaxDeg];
#pragma unroll
                for (int c = 0; c < RMAX; ++c) {
                    // idle slots read their last column's words (valid addresses)
#pragma unroll
                    for (int e = 0; e < kMaxDeg; ++e)
                        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(wn[c][e]) : "r"(nw[c][e]) : "memory");
                    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(uu[c]) : "r"(sbc[c] + lofs) : "memory");
                }
#pragma unroll
                for (int c = 0; c < RMAX; ++c) {
                    const bool act = unsigned(l - lv[c]) < unsigned(M);
                    // bit t of every column word (neighbours store M bits), bits
                    // t -/+ 1 of the own word (M-periodic, so the rotation wraps)
                    const uint32_t m = mrot[c];
                    const uint32_t mp = __funnelshift_r(m, m, 1), mn = mnext[c];
                    int fa = cq[c], fb = 0;
#pragma unroll
                    for (int e = 0; e < kMaxDeg; e += 2) {
                        fa += (wn[c][e] & m) ? nj[c][e] : 0;
                        fb += (wn[c][e + 1] & m) ? nj[c][e + 1] : 0;
                    }
                    if constexpr (LONG) {  // at a word's edges the Trotter bit is in the next word
                        fa += ((m == 1u ? wprev[c] : bits[c]) & mp) ? jt2[c] : 0;
                        fb += ((m == 0x80000000u ? wnext[c] : bits[c]) & mn) ? jt2[c] : 0;
                    } else {
                        fa += (bits[c] & mp) ? jt2[c] : 0;
                        fb += (bits[c] & mn) ? jt2[c] : 0;
                    }
                    const int h = fa + fb;                 // the local field
                    const int k = (bits[c] & m) ? h : -h;  // s_t f
                    // T(k) for 0 < k < K (lane k), else T(0) = 0: flip iff k <= 0
                    // or u < T(k).  Lane index min(k, 32) as unsigned: lanes K ..
                    // 31 hold 0, and 32 (k < 0 or k >= 32) wraps to lane 0.
                    uint32_t th;
                    if (shfl_thr)
                        th = __shfl_sync(FULL, thr_lane, min(unsigned(k), 32u));
                    else
                        th = unsigned(k - 1) < unsigned(K - 1) ? thr_s[k] : 0u;
                    const bool take = act && (k <= 0 || uu[c] < th);
                    bits[c] ^= take ? m : 0u;
                    dk += take ? k : 0;
                    asm volatile("{ .reg .pred p; setp.ne.b32 p, %2, 0; @p st.shared.u32 [%0], %1; }" ::"r"(sa[c]),
                                 "r"(bits[c] & cmask), "r"(take ? 1u : 0u)
                                 : "memory");
                }
            }  // any
            if constexpr (LONG) {
                // a busy slot at the last slice of a word moves to the next word (S
                // words further on):
                // its neighbours' words too; the next word is word 0 when
                // entering the column's last word (slice M - 1's ring neighbour)
#pragma unroll
                for (int c = 0; c < RMAX; ++c) {
                    const int t = l - lv[c];
                    if (mrot[c] == 0x80000000u && t >= 0 && t < M - 1) {
                        const uint32_t wstride = 4u * uint32_t(S);  // bytes between a column's words
                        wprev[c] = bits[c];
                        bits[c] = wnext[c];
                        sa[c] += wstride;
#pragma unroll
                        for (int e = 0; e < kMaxDeg; ++e)
                            nw[c][e] += wstride;
                        asm volatile("ld.shared.u32 %0, [%1];"
                                     : "=r"(wnext[c])
                                     : "r"(t + 33 < M ? sa[c] + wstride : sa0[c])
                                     : "memory");
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < RMAX; ++c)
                mrot[c] = mnext[c];
            // the word stream
            if (ring_words) {
                if (PH == 0)
                    fetch_words(wsw, l);
            } else {
                if (PH == 0) {
                    philox_start(sid, l, false);
                } else {
#pragma unroll
                    for (int c = 0; c < RMAX; ++c) {
                        if (pgo[c]) {
#pragma unroll
                            for (int i = 0; i < 3; ++i)
                                if (PH < 3 || i == 0)
                                    philox_round(pc[c], pk0[c], pk1[c]);
                            if (PH == 3)
                                philox_store(c);
                        }
                    }
                }
            }
            // the level barrier of the sweep threads
            asm volatile("bar.sync 1, %0;" ::"r"(T) : "memory");
        };
        for (int l = 0; l < a.D; l += 4) {
            level(l, std::integral_constant<int, 0>{});
            if (l + 1 < a.D)
                level(l + 1, std::integral_constant<int, 1>{});
            if (l + 2 < a.D)
                level(l + 2, std::integral_constant<int, 2>{});
            if (l + 3 < a.D)
                level(l + 3, std::integral_constant<int, 3>{});
        }
        __syncthreads();  // sweep end (block-wide): the generator has the next sweep's words

        // slots back at their first column; the next sweep's first blocks
        // requested, in flight during PT
        restart();
        if (ring_words && sw + 1 < a.nsweeps) {
            const uint32_t* wn = gen ? gen_buf(sw + 1) : wsw + a.wbuf_sweep_stride;
            request_words(wn, -8);
            request_words(wn, -4);
        }
        }  // sweep threads

        if (fused && (sw + 1) % a.swap_every == 0) {
            {  // one shared atomic per warp
                const int wsum = __reduce_add_sync(FULL, dk);
                if ((tid & 31) == 0 && wsum != 0)
                    atomicAdd(&eacc[0], 2 * wsum);
            }
            dk = 0;
            const unsigned long long p = pass0 + npass;
            const int par = int(p & 1ull);
            // the pass moves this replica's temperature t at most to its pair
            // partner: both threshold rows are loaded before the barrier
            const int t_old = temp_s[r];
            const int t_alt = ((t_old - par) & 1) == 0 ? t_old + 1 : t_old - 1;
            uint32_t th_old = 0u, th_alt = 0u;
            if (shfl_thr && (tid & 31) < K) {
                th_old = __ldg(a.thr + size_t(t_old) * K + (tid & 31));
                if (t_alt >= 0 && t_alt < R)
                    th_alt = __ldg(a.thr + size_t(t_alt) * K + (tid & 31));
            }
            // this thread's first pair: its table row and (MT19937) swap word do
            // not depend on the energies, so they are loaded before the barrier
            const int npairs = par ? (R - 1) / 2 : R / 2;
            int pre_len = 0, pre_off = 0;
            uint32_t pre_u = 0u;
            if (tid < npairs) {
                pre_len = a.swlen[2 * tid + par];
                pre_off = a.swoff[2 * tid + par];
                if (RNG == 0)
                    pre_u = a.swbuf[size_t(npass) * a.maxpairs + tid];
            }
            __syncthreads();
            int* Ep = a.E_pub + size_t(npass & 1) * R;
            if (tid == 0) {
                const int e = a.E[r] + eacc[0];
                a.E[r] = e;
                Ep[r] = e;
                eacc[0] = 0;
            }
            if (nblk == 1)
                __syncthreads();
            else if (!grid_sync(a.gridbar, unsigned(npass + 1) * unsigned(nblk), a.err, &s_flag))
                return;
            {  // the pairs of a pass are disjoint: one per thread
                for (int j = tid; j < npairs; j += NT) {
                    const int k = 2 * j + par;
                    const bool first = j == tid;
                    const int sa = slot_s[k], sb = slot_s[k + 1];
                    const long long d = (long long)__ldcg(Ep + sa) - (long long)__ldcg(Ep + sb);
                    uint32_t u;
                    if (RNG == 0)
                        u = first ? pre_u : a.swbuf[size_t(npass) * a.maxpairs + j];
                    else
                        u = pick4(philox4x32_10(make_uint4(uint32_t(j) >> 2, uint32_t(p), a.inst, 1u), a.seed,
                                                0xFFFFFFFFu),
                                  j & 3);
                    const int len = first ? pre_len : a.swlen[k], off = first ? pre_off : a.swoff[k];
                    const bool take = (d <= 0) || (d < len && u < a.swthr[off + d]);
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
            if (shfl_thr) {
                thr_lane = temp_s[r] == t_old ? th_old : th_alt;
            } else {
                for (int k = tid; k < K; k += NT)
                    thr_s[k] = a.thr[size_t(temp_s[r]) * K + k];
                __syncthreads();
            }
            ++npass;
        }
    }
    if (ring_words)
        asm volatile("cp.async.wait_all;" ::: "memory");
    if (RNG == 0 && is_gen) {  // the stream as it now stands
        gen_sync();
        for (int i = glane; i < kMtRing; i += GL)
            a.mtring[size_t(r) * kMtRing + i] = gring[i];
        if (glane == 0)
            a.mtpos[r] += (unsigned long long)a.nsweeps * (unsigned long long)N;
    }

    // ---- energies and write-back (coalesced over the spin index)
    {
        const int wsum = __reduce_add_sync(FULL, dk);
        if ((tid & 31) == 0 && wsum != 0)
            atomicAdd(&eacc[0], 2 * wsum);
    }
    __syncthreads();
    if (tid == 0)
        a.E[r] += eacc[0];
    int8_t* spo = a.spins + size_t(r) * N;
    for (int i = tid; i < N; i += NT) {
        const int t = i / S, q = i - t * S, p = pos[q];
        const int tm = (t == 0) ? M - 1 : t - 1, tp = (t == M - 1) ? 0 : t + 1;
        const uint32_t* d = desc + p * kDescWords;
        const int wo = LONG ? (t >> 5) : 0;  // the word of slice t (LONG)
        const int bt = LONG ? (t & 31) : t;
        const uint32_t* cw = colw + ((d[1] - colw_s) >> 2);
        const uint32_t cb = cw[wo * S];
        const uint32_t cbm = LONG ? cw[(tm >> 5) * S] : cb, cbp = LONG ? cw[(tp >> 5) * S] : cb;
        int f = int(d[3]) + int(d[2]) * int(((cbm >> (LONG ? (tm & 31) : tm)) & 1u) +
                                            ((cbp >> (LONG ? (tp & 31) : tp)) & 1u));
        for (int e = 0; e < kMaxDeg; ++e)
            f += int(d[10 + e]) * int((colw[((d[4 + e] - colw_s) >> 2) + wo * S] >> bt) & 1u);
        spo[i] = ((cb >> bt) & 1u) ? int8_t(1) : int8_t(-1);
        if (f16)
            static_cast<int16_t*>(a.fields)[size_t(r) * N + i] = int16_t(f);
        else
            static_cast<int*>(a.fields)[size_t(r) * N + i] = f;
    }
    if (fused && blk == 0)
        for (int i = tid; i < R; i += NT) {
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

// Register budget: about 30 registers per slot round; blocks of up to 256
// sweep threads (one round) or 128 (more rounds), plus the generator warps,
// two resident blocks per SM.
template <int RNG, int RMAX, bool LONG = false>
__global__ void __launch_bounds__(RMAX == 1 ? 256 + 64 : 128 + 64, 2) packed_kernel(const SweepArgs a)
{
    packed_body<RNG, RMAX, LONG>(a, int(blockIdx.x), int(gridDim.x));
}

// Ragged batches: block b runs replica items[b].block of instance
// items[b].inst with that instance's arguments (copied to shared memory), all
// sweeps of the launch with the instance's PT passes fused; a launch holds
// whole instances, all of its blocks resident (cooperative launch), and the
// instances' grid-barrier counters start at zero.
template <int RNG, int RMAX>
__global__ void __launch_bounds__(RMAX == 1 ? 256 + 64 : 128 + 64, 2)
    packed_batch_kernel(const SweepArgs* __restrict__ args, const BatchItem* __restrict__ items)
{
    __shared__ SweepArgs sa;
    const BatchItem it = items[blockIdx.x];
    if (threadIdx.x == 0)
        sa = args[it.inst];
    __syncthreads();
    packed_body<RNG, RMAX>(sa, it.block, sa.inst_blocks);
}

template <int RNG>
void* pick_packed_batch(int rmax)
{
    switch (rmax) {
    case 1: return reinterpret_cast<void*>(&packed_batch_kernel<RNG, 1>);
    case 2: return reinterpret_cast<void*>(&packed_batch_kernel<RNG, 2>);
    case 3: return reinterpret_cast<void*>(&packed_batch_kernel<RNG, 3>);
    default: return nullptr;
    }
}

template <int RNG>
void* pick_packed(int rmax)
{
    switch (rmax) {
    case 1: return reinterpret_cast<void*>(&packed_kernel<RNG, 1>);
    case 2: return reinterpret_cast<void*>(&packed_kernel<RNG, 2>);
    case 3: return reinterpret_cast<void*>(&packed_kernel<RNG, 3>);
    case 5: return reinterpret_cast<void*>(&packed_kernel<RNG, 5>);
    case 8: return reinterpret_cast<void*>(&packed_kernel<RNG, 8>);
    // long columns (M a multiple of 32 above 32): round count + kPackedLong
    case 101: return reinterpret_cast<void*>(&packed_kernel<RNG, 1, true>);
    case 102: return reinterpret_cast<void*>(&packed_kernel<RNG, 2, true>);
    default: return nullptr;
    }
}

}  // namespace packed_detail

// slot rounds per thread with an instantiation, and the kernels (packed_mt.cu,
// packed_philox.cu)
constexpr int kPackedRounds[5] = {1, 2, 3, 5, 8};
constexpr int kPackedLong = 100;  // round codes of the long-column instantiations: 100 + rounds (1, 2)
constexpr int kPackedGenWarps = packed_detail::kGenWarps;
void* packed_kernel_mt(int rmax, bool batch = false);
void* packed_kernel_philox(int rmax, bool batch = false);
inline void* packed_kernel_ptr(int rng, int rmax, bool batch = false)
{
    return rng == 0 ? packed_kernel_mt(rmax, batch) : packed_kernel_philox(rmax, batch);
}
size_t packed_smem_bytes(const SweepArgs& a, int threads);

}  // namespace isg
