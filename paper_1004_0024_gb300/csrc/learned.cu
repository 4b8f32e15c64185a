// Learned Trotter-column proposal with an exact Metropolis-Hastings correction
// (not in the paper; built on its layered QMC models, section 3.1).
//
// Network 33 -> 256 -> 256 -> 32 (inputs phi_t/8 for the M <= 32 slices of a
// column and beta; ReLU; outputs the logits of P(s'_t = +1)).  All dense
// layers run on the tcgen05 GEMM (tc_gemm.cu) with bf16 operands and FP32
// accumulation; FP32 master weights are trained with Adam on the mean
// Bernoulli negative log-likelihood of columns sampled by the plain sweep.
//
// A learned pass visits the slice graph's colour classes (greedy colouring:
// columns of one class share no spatial edge, so their conditional laws do
// not interact) and, for every replica and column of a class: gathers phi
// from the spins, evaluates the network, draws s'_t = +1 iff u_t < p_t 2^32,
// and accepts with probability min(1, exp(-beta dE + log q(s) - log q(s'))),
// dE the exact integer change of the column energy.  Both log q terms are
// the exact probabilities of the discrete draw actually made (FP64), so the
// move leaves the Boltzmann law invariant whatever the network's precision.
// Energies are updated by dE; local fields incrementally: a moved column's
// own fields are phi_t plus its new Trotter neighbours, and every flipped
// spin moves its spatial neighbours' fields by 2 J s' (atomically: two
// columns of a class may share a neighbour).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <set>
#include <vector>

#include "handle.h"
#include "ising_internal.cuh"

using bf16 = __nv_bfloat16;

namespace isg {
namespace {

constexpr int kHid = 256;  // hidden width
constexpr int kIn = 64;    // padded input width (M + 1 <= 33 used)
constexpr int kOut = 32;   // padded output width (M used)

__global__ void gather_batch_kernel(const bf16* __restrict__ Xd, const uint32_t* __restrict__ Yd,
                                    const int* __restrict__ idx, int B, bf16* __restrict__ Xb,
                                    uint32_t* __restrict__ Yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (row, 16-byte chunk)
    if (i >= B * (kIn / 8))
        return;
    const int row = i / (kIn / 8), c = i % (kIn / 8);
    const long long src = idx[row];
    reinterpret_cast<uint4*>(Xb + size_t(row) * kIn)[c] = reinterpret_cast<const uint4*>(Xd + size_t(src) * kIn)[c];
    if (c == 0)
        Yb[row] = Yd[src];
}

__device__ __forceinline__ float softplusf(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

// dL = (sigmoid(l) - y) / B as a bf16 pair: dL[b][j] = hi, dL[b][32 + j] = lo
// with hi + lo = the FP32 value to 16 bits (the GEMMs against W3 see W3 twice
// along K, so they use hi + lo); 0 for the padding; loss += BCE.
__global__ void bce_kernel(const float* __restrict__ L, const uint32_t* __restrict__ Y, int B, int out,
                           float inv_b, bf16* __restrict__ dL, float* __restrict__ loss)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.f;
    if (b < B) {
        const uint32_t y = Y[b];
        for (int j = 0; j < kOut; ++j) {
            float d = 0.f;
            if (j < out) {
                const float l = L[size_t(b) * kOut + j];
                const float t = float((y >> j) & 1u);
                acc += softplusf(l) - t * l;
                d = (1.f / (1.f + expf(-l)) - t) * inv_b;
            }
            const bf16 hi = __float2bfloat16(d);
            dL[size_t(b) * kIn + j] = hi;
            dL[size_t(b) * kIn + kOut + j] = __float2bfloat16(d - __bfloat162float(hi));
        }
    }
    __shared__ float red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        atomicAdd(loss, red[0]);
}

// gW3 += its lo half (rows 32..63 of the GEMM output), gb3 = hi + lo sums
__global__ void fold_kernel(float* __restrict__ gW3, float* __restrict__ gb3, const float* __restrict__ cs64)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kOut * kHid)
        gW3[i] += gW3[kOut * kHid + i];
    if (i < kOut)
        gb3[i] = cs64[i] + cs64[kOut + i];
}

// dst[c][r] = src[r][c] for r < rows, c < cols (32 x 32 tiles through shared memory)
__global__ void transpose_kernel(const bf16* __restrict__ src, int rows, int cols, int lds,
                                 bf16* __restrict__ dst, int ldd)
{
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = r0 + y, c = c0 + threadIdx.x;
        if (r < rows && c < cols)
            tile[y][threadIdx.x] = src[size_t(r) * lds + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = c0 + y, r = r0 + threadIdx.x;
        if (r < rows && c < cols)
            dst[size_t(c) * ldd + r] = tile[threadIdx.x][y];
    }
}

// out[c] = sum_r src[r][c]
__global__ void colsum_kernel(const bf16* __restrict__ src, int rows, int cols, int lds, float* __restrict__ out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols)
        return;
    float a = 0.f;
    for (int r = 0; r < rows; ++r)
        a += __bfloat162float(src[size_t(r) * lds + c]);
    out[c] = a;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
}

// dst = bf16(src) for a [rows][cols] matrix, optionally transposed into [cols][ldd]
__global__ void to_bf16_kernel(const float* __restrict__ src, int rows, int cols, bf16* __restrict__ dst,
                               int ldd, int transpose)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols)
        return;
    const int r = i / cols, c = i % cols;
    const bf16 v = __float2bfloat16(src[i]);
    if (transpose)
        dst[size_t(c) * ldd + r] = v;
    else
        dst[size_t(r) * ldd + c] = v;
}

// dst = bf16(src) for a [rows][cols] matrix in the tiled operand layout of
// the fused network kernel (tiled_offset with `rows` rows)
__global__ void tile_bf16_kernel(const float* __restrict__ src, int rows, int cols, unsigned char* __restrict__ dst)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols)
        return;
    const int r = i / cols, c = i % cols;
    *reinterpret_cast<bf16*>(dst + tiled_offset(rows, r, c)) = __float2bfloat16(src[i]);
}

}  // namespace
}  // namespace isg

namespace isg {
namespace {

struct LearnedArgs {
    int S, M, N, R, rows, ncols;  // rows = R * ncols (real rows of this class)
    const int *row_ptr, *col, *J, *h, *jtau, *pos;
    int8_t* spins;
    int* E;
    const int* temp_of_slot;
    const double* betas;
    const float* betas32;
    const int* sites;  // the class's sites
    const int* sp_off; // [S+1] spatial neighbour list of each site
    const int2* sp_nbr; // (site, J) entries
    uint32_t* colbits;  // [R][S] column bits: bit t = (spin (t, q) > 0)
    int sp_simd;        // every site has sum_j 2 |J_qj| <= 127 (byte-lane phi)
    int* phi;          // [rows][32]
    bf16* X;           // rows_pad x 64 inputs, in tiles of 128 rows in the operand layout
    const float* L;    // [rows_pad / 128][32][128]: logit t of row i at (i / 128, t, i % 128)
    uint32_t seed, inst, pass;
    uint32_t *old_bits, *prop_bits;
    uint32_t* acc_word;  // [rows] the acceptance word of each row (Philox word 32)
    uint8_t* accepted;
    unsigned long long* n_acc;
    unsigned long long* n_exact;  // decisions taken by the FP64 product
    unsigned long long* n_changed;  // accepted moves with s' != s
    int fp64_only;                // decide every move by the FP64 product
    int mixture;                  // flip-symmetric mixture (q(s') + q(-s')) / 2
    void* fields;                 // [R][N] local fields, int16 or int32
    int field_bits;
};

// phi_t = h_i + sum over spatial neighbours j (same slice) of J s_j, i = t S + q
__device__ __forceinline__ int spatial_field(const LearnedArgs& a, const int8_t* sp, int t, int q)
{
    const int i = t * a.S + q;
    int f = a.h[i];
    for (int e = a.row_ptr[i]; e < a.row_ptr[i + 1]; ++e) {
        const int j = a.col[e];
        if (j / a.S == t)
            f += a.J[e] * int(sp[j]);
    }
    return f;
}

// Trotter part of the local field of slice t of a column: Jtau (s_{t-1} +
// s_{t+1}) on the ring (M >= 3), Jtau s_{1-t} for M == 2, 0 for M == 1
__device__ __forceinline__ int column_trotter(uint32_t bits, int t, int M, int jt)
{
    if (M == 1)
        return 0;
    const int tp = (t + 1 == M) ? 0 : t + 1;
    const int sp = ((bits >> tp) & 1u) ? 1 : -1;
    if (M == 2)
        return jt * sp;
    const int tm = (t == 0) ? M - 1 : t - 1;
    return jt * (sp + (((bits >> tm) & 1u) ? 1 : -1));
}

// Column bits of every (replica, site) from the spins: bit t = (s_(t, q) > 0).
// Thread per column; for each slice the lanes read consecutive bytes.
__global__ void __launch_bounds__(256) learned_colbits_kernel(const LearnedArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // k = r S + q
    if (k >= a.R * a.S)
        return;
    const int r = k / a.S, q = k - r * a.S;
    const int8_t* sp = a.spins + size_t(r) * a.N + q;
    uint32_t bits = 0u;
#pragma unroll
    for (int t = 0; t < kOut; ++t)
        if (t < a.M)
            bits |= uint32_t(sp[size_t(t) * a.S] > 0) << t;
    a.colbits[k] = bits;
}

// phi_t = h_q + sum over the spatial neighbours j of site q of J_qj s_(t, j)
// for t < 32 (every slice holds the same h and couplings), from the column
// bits of replica r's neighbours: s = 2 b - 1, so phi_t = h_q - sum_j J_qj +
// sum_j 2 J_qj b_j(t).  The last sum is kept in byte lanes, four slices per
// 32-bit word starting at 128 per byte: each neighbour spreads four of its
// bits to the low bit of four bytes (x * 0x00204081 & 0x01010101) and adds
// 2 J times that.  Every partial sum stays within 128 -+ sum_j 2 |J_qj|, so
// with that bound at most 127 (checked on the host: simd) no byte carries or
// borrows into the next.  Otherwise the sum is formed slice by slice.
__device__ __forceinline__ void column_phi(const LearnedArgs& a, const uint32_t* cb, int q, int (&f)[kOut])
{
    int base = a.h[q];
    const int e0 = a.sp_off[q], e1 = a.sp_off[q + 1];
    if (a.sp_simd) {
        uint32_t acc[kOut / 4];
#pragma unroll
        for (int w = 0; w < kOut / 4; ++w)
            acc[w] = 0x80808080u;
        for (int e = e0; e < e1; ++e) {
            const int2 nb = a.sp_nbr[e];
            const uint32_t b = cb[nb.x];
            const uint32_t j2 = uint32_t(2 * nb.y);
            base -= nb.y;
#pragma unroll
            for (int w = 0; w < kOut / 4; ++w)
                acc[w] += ((((b >> (4 * w)) & 0xFu) * 0x00204081u) & 0x01010101u) * j2;
        }
#pragma unroll
        for (int t = 0; t < kOut; ++t)
            f[t] = base - 128 + int((acc[t >> 2] >> (8 * (t & 3))) & 0xFFu);
        return;
    }
#pragma unroll
    for (int t = 0; t < kOut; ++t)
        f[t] = 0;
    for (int e = e0; e < e1; ++e) {
        const int2 nb = a.sp_nbr[e];
        const uint32_t b = cb[nb.x];
        const int j2 = 2 * nb.y;
        base -= nb.y;
#pragma unroll
        for (int t = 0; t < kOut; ++t)
            f[t] += ((b >> t) & 1u) ? j2 : 0;
    }
#pragma unroll
    for (int t = 0; t < kOut; ++t)
        f[t] += base;
}

// One thread per (replica, column) row: phi of the column from the current
// column bits (the moves of earlier classes are seen without any field being
// maintained during the pass), then the input row X = (phi_t/8 for t < M,
// beta at M, zeros) in the tiled operand layout of the fused network, 16
// bytes (8 inputs) at a time, and the column's bits to old_bits.
__global__ void __launch_bounds__(128) learned_gather_kernel(const LearnedArgs a, int rows_pad)
{
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows_pad)
        return;
    unsigned char* xt = reinterpret_cast<unsigned char*>(a.X) + size_t(row >> 7) * (128 * 128);
    const int rt = row & 127;
    if (row >= a.rows) {
#pragma unroll
        for (int k0 = 0; k0 < 64; k0 += 8)
            *reinterpret_cast<uint4*>(xt + tiled_offset(128, rt, k0)) = make_uint4(0u, 0u, 0u, 0u);
        return;
    }
    const int r = row / a.ncols, q = a.sites[row - r * a.ncols];
    const int M = a.M;
    const uint32_t* cb = a.colbits + size_t(r) * a.S;
    int f[kOut];
    column_phi(a, cb, q, f);
    const float beta = a.betas32[a.temp_of_slot[r]];
    int* phi = a.phi + size_t(row) * kOut;
#pragma unroll
    for (int k0 = 0; k0 < 64; k0 += 8) {
        uint32_t packed[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = k0 + u + h;
                v[h] = (k < kOut && k < M) ? float(f[k < kOut ? k : 0]) * 0.125f : (k == M ? beta : 0.f);
            }
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[0], v[1]);
            packed[u >> 1] = *reinterpret_cast<const uint32_t*>(&b2);
        }
        *reinterpret_cast<uint4*>(xt + tiled_offset(128, rt, k0)) =
            make_uint4(packed[0], packed[1], packed[2], packed[3]);
        if (k0 < kOut) {
            *reinterpret_cast<int4*>(phi + k0) = make_int4(f[k0], f[k0 + 1], f[k0 + 2], f[k0 + 3]);
            *reinterpret_cast<int4*>(phi + k0 + 4) = make_int4(f[k0 + 4], f[k0 + 5], f[k0 + 6], f[k0 + 7]);
        }
    }
    a.old_bits[row] = cb[q];
    // word 32 of the row (block 8, counter 2 + 32), drawn here where the
    // issue slots are idle behind the loads
    a.acc_word[row] = philox4x32_10(make_uint4(uint32_t(q), a.pass, a.inst, 34u), a.seed, uint32_t(r)).x;
}

// Local fields of every spin after a pass: f_(t,q) = phi_t of column q plus
// its Trotter part J_tau (s_(t-1,q) + s_(t+1,q)) on the ring (J_tau s_(1-t,q)
// for M == 2, none for M == 1).  Thread per (replica, column); for each slice
// the lanes write consecutive fields.
template <typename F>
__global__ void __launch_bounds__(256) learned_fields_kernel(const LearnedArgs a)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // k = r S + q
    if (k >= a.R * a.S)
        return;
    const int r = k / a.S, q = k - r * a.S;
    const uint32_t* cb = a.colbits + size_t(r) * a.S;
    int f[kOut];
    column_phi(a, cb, q, f);
    const uint32_t bits = cb[q];
    const int jt = a.jtau[a.pos[q]];
    F* fl = static_cast<F*>(a.fields) + size_t(r) * a.N + q;
#pragma unroll
    for (int t = 0; t < kOut; ++t)
        if (t < a.M)
            fl[size_t(t) * a.S] = F(f[t] + column_trotter(bits, t, a.M, jt));
}

// Term of slice t in E_col: -s_t phi_t - Jtau s_t s_{t+1 mod M} (the Trotter
// term on every slice for M >= 3, on slice 0 only for M == 2, none for M == 1)
__device__ __forceinline__ int column_term(uint32_t bits, int t, int M, int phi, int jt)
{
    const int s = ((bits >> t) & 1u) ? 1 : -1;
    int e = -s * phi;
    if (M >= 3 || (M == 2 && t == 0)) {
        const int t1 = (t + 1 == M) ? 0 : t + 1;
        e -= jt * s * (((bits >> t1) & 1u) ? 1 : -1);
    }
    return e;
}

// c_t = ceil(p_t 2^32) of slice t's logit, p_t = 1 / (1 + exp(-l)) in FP32,
// as an FP32 value: p 2^32 is exact (a power-of-two scale) and so is its
// ceiling (every integer below 2^24 is a float, and above 2^24 p 2^32 is
// already an integer), so c is the integer ceil(p 2^32) exactly, at most 2^32
__device__ __forceinline__ float proposal_c(float l)
{
    return ceilf(1.f / (1.f + expf(-l)) * 4294967296.f);
}

// The mixture mode keeps every slice's probability strictly inside (0, 1):
// c clamped to [1, 2^32 - 1] (integers, exact in FP32 up to 2^24 and, above,
// 2^32 - 256 is the largest float below 2^32), so that log q is finite for
// every column
__device__ __forceinline__ float proposal_c_mix(float l)
{
    return fminf(fmaxf(proposal_c(l), 1.f), 4294967040.f);
}

// u < c for a 32-bit word u and an integer-valued c in [0, 2^32]
__device__ __forceinline__ bool word_below(uint32_t u, float c)
{
    return c >= 4294967296.f || u < uint32_t(c);
}

// One MH column move per group of 8 lanes (kMhLanes): lane g of the group
// draws Philox block g, proposes slices 4g .. 4g+3 and adds their terms; the
// group combines bits and sums by shuffles (word 32 was drawn by the gather).  Words: Philox4x32-10, key
// (seed, r), counter (q, pass, instance, 2 + 4 j) gives words 4j .. 4j+3;
// word t < M proposes slice t, word 32 decides acceptance.  Bit t is drawn +1
// iff u_t < p_t 2^32 (p_t the FP32 sigmoid of the logit), i.e. iff u_t < c_t
// with c_t = ceil(p_t 2^32): an event of probability exactly c_t 2^-32.  The
// Hastings ratio q(s)/q(s') is the product over the changed bits of
// c(old bit) / c(new bit) (c(+1) = c_t, c(-1) = 2^32 - c_t), formed in FP64
// with exact exponents, so it is the ratio of the probabilities of the draws
// actually made.  An FP32 estimate of its logarithm, with a bound on its
// error, decides whenever the bound allows.
//
// Mixture (flip-symmetric) proposal q_mix(s') = (q(s') + q(-s')) / 2: the
// sign bit of word 33 (Philox block 34's second word) chooses q's draw or its
// complement.  With kappa_t = log(c_t / (2^32 - c_t)) and K(x) = sum_t x_t
// kappa_t (x_t = +-1), log q(-x) - log q(x) = -K(x), so
//     log q_mix(s) - log q_mix(s') = log q(s) - log q(s')
//                                    + softplus(-K(s)) - softplus(-K(s')),
// the first part the ratio above, the rest summed over all M slices (FP32
// with its error bound, FP64 when the bound cannot decide).  In this mode c_t
// is clamped to [1, 2^32 - 256] (proposal_c_mix), so every kappa is finite.
constexpr int kMhLanes = 8;
constexpr int kMhThreads = 256;
constexpr int kMhRows = kMhThreads / kMhLanes;  // rows per block

__global__ void __launch_bounds__(kMhThreads) learned_mh_kernel(const LearnedArgs a)
{
    __shared__ unsigned s_cnt[2][kMhThreads / 32];
    __shared__ int s_dE[kMhRows + 2];  // energy change per replica of the block's rows
    const int r0 = int(blockIdx.x) * kMhRows / a.ncols;
    const int nrep = min((int(blockIdx.x) * kMhRows + kMhRows - 1) / a.ncols, a.R - 1) - r0 + 1;
    for (int k = threadIdx.x; k < nrep; k += blockDim.x)
        s_dE[k] = 0;
    __syncthreads();
    const int row = int(blockIdx.x) * kMhRows + int(threadIdx.x) / kMhLanes;
    const int g = threadIdx.x & (kMhLanes - 1);
    const unsigned gmask = 0xFFu << (threadIdx.x & 24);  // the lanes of this row's group
    bool acc = false, moved = false;
    if (row < a.rows) {  // uniform over the group
        const int r = row / a.ncols, q = a.sites[row - r * a.ncols];
        const int M = a.M, S = a.S;
        const uint32_t old = a.old_bits[row];
        const float* Lr = a.L + size_t(row >> 7) * (128 * kOut) + (row & 127);  // logit t at Lr[128 t]
        const int jt = a.jtau[a.pos[q]];
        const bool live = 4 * g < M;
        uint32_t prop = 0u;
        float lq = 0.f, mag = 0.f;
        float ks = 0.f, ks2 = 0.f, magk = 0.f;  // mixture: K(s), K(s'), sum |kappa|
        bool flip = false;                       // mixture: the complement of q's draw
        if (a.mixture) {
            uint32_t bw = 0u;
            if (g == 0)
                bw = philox4x32_10(make_uint4(uint32_t(q), a.pass, a.inst, 34u), a.seed, uint32_t(r)).y;
            flip = (__shfl_sync(gmask, bw, threadIdx.x & 24) >> 31) != 0u;
        }
        if (live) {
            const uint4 w = philox4x32_10(make_uint4(uint32_t(q), a.pass, a.inst, 2u + 4u * uint32_t(g)), a.seed,
                                          uint32_t(r));
            const uint32_t wv[4] = {w.x, w.y, w.z, w.w};
            float lv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                lv[u] = Lr[size_t(4 * g + u) * 128];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 4 * g + u;
                if (t < M) {
                    const float c1 = a.mixture ? proposal_c_mix(lv[u]) : proposal_c(lv[u]);
                    const bool up = word_below(wv[u], c1) != flip;
                    const bool ob = (old >> t) & 1u;
                    prop |= uint32_t(up) << t;
                    if (up != ob) {  // FP32 log of this bit's ratio
                        const float cp = c1, cm = 4294967296.f - c1;  // cm: 2^32 - c rounded once
                        const float term = logf(up ? cm / cp : cp / cm);
                        lq += term;
                        mag += fabsf(term);
                    }
                    if (a.mixture) {
                        const float kap = logf(c1 / (4294967296.f - c1));
                        ks += ob ? kap : -kap;
                        ks2 += up ? kap : -kap;
                        magk += fabsf(kap);
                    }
                }
            }
        }
#pragma unroll
        for (int o = kMhLanes / 2; o > 0; o >>= 1) {
            prop |= __shfl_xor_sync(gmask, prop, o);
            lq += __shfl_xor_sync(gmask, lq, o);
            mag += __shfl_xor_sync(gmask, mag, o);
            ks += __shfl_xor_sync(gmask, ks, o);
            ks2 += __shfl_xor_sync(gmask, ks2, o);
            magk += __shfl_xor_sync(gmask, magk, o);
        }
        int dE = 0;
        if (live) {
            const int4 p4 = *reinterpret_cast<const int4*>(a.phi + size_t(row) * kOut + 4 * g);
            const int pv[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 4 * g + u;
                if (t < M)
                    dE += column_term(prop, t, M, pv[u], jt) - column_term(old, t, M, pv[u], jt);
            }
        }
#pragma unroll
        for (int o = kMhLanes / 2; o > 0; o >>= 1)
            dE += __shfl_xor_sync(gmask, dE, o);
        if (g == 0) {
            const uint32_t ua = a.acc_word[row];
            const float bdE = a.betas32[a.temp_of_slot[r]] * float(dE);
            auto softplus32 = [](float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); };
            const float sp1 = a.mixture ? softplus32(-ks) : 0.f, sp2 = a.mixture ? softplus32(-ks2) : 0.f;
            const float lmix = sp1 - sp2;
            const float la = -bdE + lq + lmix;
            const float lu = logf((float(ua) + 0.5f) * 2.3283064365386963e-10f);
            // Bound on |la - logA| + |lu - log u'|: each term's ratio carries 3
            // roundings (1.8e-7 in the log, 5.8e-6 over 32 terms) and logf 1
            // ulp (1.2e-7 |term|); the sums at most 31 roundings (1.9e-6 mag);
            // beta, the product and the sum 1.8e-7 |bdE|; lu 2.9e-6.  Below
            // 8.7e-6 + 1.8e-7 |bdE| + 2.1e-6 mag.  Mixture: each kappa carries
            // 2 roundings and logf 1 ulp (1.2e-7 + 1.2e-7 |kappa|), each K sum
            // at most 31 roundings, so |K - K_exact| <= eK = 3.9e-6 + 2e-6 magk;
            // softplus(-K) moves by at most eK sigma(-(K - eK)) (its slope is
            // sigma(-K), decreasing in K), taken 1% high, plus its own FP32
            // rounding (expf, log1pf, the add) below 1e-6 (1 + its value); the
            // difference and the last sum 2e-7 |lmix| + 1e-7.
            float eps = 1e-5f * (1.f + fabsf(bdE) + mag);
            if (a.mixture) {
                const float eK = 3.9e-6f + 2e-6f * magk;
                const float sg = 1.f / (1.f + expf(ks - eK)) + 1.f / (1.f + expf(ks2 - eK));
                eps += 1.01f * eK * sg + 1e-6f * (2.f + sp1 + sp2) + 2e-7f * fabsf(lmix) + 1e-7f;
            }
            bool decided = !a.fp64_only;
            if (decided) {
                if (la >= eps || lu < la - eps)
                    acc = true;
                else if (la < -eps && lu > la + eps)
                    acc = false;
                else
                    decided = false;
            }
            if (!decided) {  // exact: the FP64 product of the integer ratios
                double num = 1.0, den = 1.0;
                int en = 0, ed = 0, n = 0;
                for (uint32_t ch = old ^ prop; ch; ch &= ch - 1u) {
                    const int b = __ffs(ch) - 1;
                    const float cb = a.mixture ? proposal_c_mix(Lr[size_t(b) * 128]) : proposal_c(Lr[size_t(b) * 128]);
                    const double cp = double(cb), cm = 4294967296.0 - cp;
                    const bool ob = (old >> b) & 1u;
                    num *= ob ? cp : cm;
                    den *= ob ? cm : cp;
                    if ((++n & 15) == 0) {  // 16 factors of <= 2^32: renormalise
                        int k;
                        num = frexp(num, &k);
                        en += k;
                        den = frexp(den, &k);
                        ed += k;
                    }
                }
                double logA = -a.betas[a.temp_of_slot[r]] * double(dE) + log(num / den) +
                              double(en - ed) * 0.6931471805599453;
                if (a.mixture) {  // + softplus(-K(s)) - softplus(-K(s')) in FP64
                    double k1 = 0.0, k2 = 0.0;
                    for (int t = 0; t < M; ++t) {
                        const double cp = double(proposal_c_mix(Lr[size_t(t) * 128]));
                        const double kap = log(cp / (4294967296.0 - cp));
                        k1 += ((old >> t) & 1u) ? kap : -kap;
                        k2 += ((prop >> t) & 1u) ? kap : -kap;
                    }
                    auto softplus64 = [](double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); };
                    logA += softplus64(-k1) - softplus64(-k2);
                }
                acc = (logA >= 0.0) || (log((double(ua) + 0.5) * 2.3283064365386963e-10) < logA);
                atomicAdd(a.n_exact, 1ull);
            }
            a.prop_bits[row] = prop;
            a.accepted[row] = acc ? 1 : 0;
            moved = acc && prop != old;
            if (moved) {  // the fields are rebuilt after the pass
                atomicAdd(&s_dE[r - r0], dE);
                a.colbits[size_t(r) * S + q] = prop;
            }
        }
        const bool mv = __shfl_sync(gmask, moved, threadIdx.x & 24);
        if (mv && live) {  // this lane's slices of the new column
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 4 * g + u;
                if (t < M && (((old ^ prop) >> t) & 1u))
                    a.spins[size_t(r) * a.N + size_t(t) * S + q] = ((prop >> t) & 1u) ? int8_t(1) : int8_t(-1);
            }
        }
    }
    const unsigned n_acc = __reduce_add_sync(0xFFFFFFFFu, acc ? 1u : 0u);
    const unsigned n_mov = __reduce_add_sync(0xFFFFFFFFu, moved ? 1u : 0u);
    if ((threadIdx.x & 31) == 0) {
        s_cnt[0][threadIdx.x >> 5] = n_acc;
        s_cnt[1][threadIdx.x >> 5] = n_mov;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned na = 0u, nm = 0u;
        for (int w = 0; w < kMhThreads / 32; ++w) {
            na += s_cnt[0][w];
            nm += s_cnt[1][w];
        }
        if (na)
            atomicAdd(a.n_acc, (unsigned long long)na);
        if (nm)
            atomicAdd(a.n_changed, (unsigned long long)nm);
    }
    for (int k = threadIdx.x; k < nrep; k += blockDim.x)
        if (s_dE[k])
            atomicAdd(&a.E[r0 + k], s_dE[k]);
}

// Training records of every (replica, column): X = (phi/8, beta), Y = spins;
// with `oriented`, Y is the column or its complement, whichever has
// sum_t s_t phi_t >= 0 (the orientation its spatial field prefers)
__global__ void collect_kernel(const LearnedArgs a, bf16* __restrict__ Xd, uint32_t* __restrict__ Yd,
                               int oriented)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;  // k = r * S + q
    if (k >= a.R * a.S)
        return;
    const int r = k / a.S, q = k - r * a.S;
    const int8_t* sp = a.spins + size_t(r) * a.N;
    bf16* x = Xd + size_t(k) * kIn;
    uint32_t y = 0u;
    long long dot = 0;
    for (int t = 0; t < a.M; ++t) {
        const int f = spatial_field(a, sp, t, q);
        x[t] = __float2bfloat16(float(f) * 0.125f);
        y |= (sp[t * a.S + q] > 0 ? 1u : 0u) << t;
        dot += (long long)f * sp[t * a.S + q];
    }
    if (oriented && dot < 0)
        y = ~y & (a.M == 32 ? 0xFFFFFFFFu : ((1u << a.M) - 1u));
    x[a.M] = __float2bfloat16(a.betas32[a.temp_of_slot[r]]);
    for (int c = a.M + 1; c < kIn; ++c)
        x[c] = __float2bfloat16(0.f);
    Yd[k] = y;
}

}  // namespace
}  // namespace isg

// ============================================================ network object
namespace {
constexpr int kW1 = isg::kHid * isg::kIn;    // [256][64], columns > M zero
constexpr int kW2 = isg::kHid * isg::kHid;   // [256][256]
constexpr int kW3 = isg::kOut * isg::kHid;   // [32][256], rows >= M zero
constexpr int kPar = kW1 + isg::kHid + kW2 + isg::kHid + kW3 + isg::kOut;
constexpr int kGW3 = 128 * isg::kHid;        // GEMM output rows are padded to 128
constexpr int kGrad = kW1 + isg::kHid + kW2 + isg::kHid + kGW3 + isg::kOut;
}  // namespace

struct ising_mlp_s {
    int M = 1;
    uint32_t seed = 0;
    cudaStream_t stream = nullptr;
    float* par = nullptr;   // W1 b1 W2 b2 W3 b3 (FP32 master copy)
    float* mom = nullptr;   // Adam first then second moments, same layout
    float* grad = nullptr;  // gW1 gb1 gW2 gb2 gW3[128][256] gb3
    long long adam_t = 0;
    bf16 *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W2tb = nullptr, *W3tb = nullptr;
    unsigned char *W1t = nullptr, *W2t = nullptr, *W3t = nullptr;  // tiled for the fused kernel
    // recorded columns
    bf16* Xd = nullptr;
    uint32_t* Yd = nullptr;
    long long cap = 0, n_rec = 0;
    int* idx = nullptr;  // [cap] shuffled record order
    // training batch workspace, sized for Bcap rows
    int Bcap = 0;
    bf16 *Xb = nullptr, *H1 = nullptr, *H2 = nullptr, *dL = nullptr, *dH2 = nullptr, *dH1 = nullptr;
    bf16 *XT = nullptr, *H1T = nullptr, *H2T = nullptr, *dLT = nullptr, *dH2T = nullptr, *dH1T = nullptr;
    float* L = nullptr;
    uint32_t* Yb = nullptr;
    float* loss = nullptr;
    float* cs64 = nullptr;  // column sums of the hi/lo output gradient
    int* err = nullptr;
    unsigned long long* n_acc = nullptr;
    // learned-pass workspace, sized for Pcap rows
    long long Pcap = 0;
    bf16* PX = nullptr;
    float* PL = nullptr;
    int* Pphi = nullptr;
    uint32_t *Pold = nullptr, *Pprop = nullptr, *Pua = nullptr;
    uint8_t* Pacc = nullptr;

    // profiling of the fused network kernel in learned passes
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    std::vector<long long> ev_rows;
    long long prof_launches = 0, prof_rows = 0;
    double prof_ms = 0.0;

    float* W1() { return par; }
    float* b1() { return par + kW1; }
    float* W2() { return b1() + isg::kHid; }
    float* b2() { return W2() + kW2; }
    float* W3() { return b2() + isg::kHid; }
    float* b3() { return W3() + kW3; }
    float* gW1() { return grad; }
    float* gb1() { return grad + kW1; }
    float* gW2() { return gb1() + isg::kHid; }
    float* gb2() { return gW2() + kW2; }
    float* gW3() { return gb2() + isg::kHid; }
    float* gb3() { return gW3() + kGW3; }
};

namespace isg {
namespace {

int32_t cuda_err(cudaError_t e, const char* what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return isg_fail(e == cudaErrorMemoryAllocation ? ISING_ERR_OOM : ISING_ERR_CUDA, m.c_str());
}

#define LCK(call)                                  \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess)                     \
            return cuda_err(e_, #call);            \
    } while (0)

template <typename T>
cudaError_t zalloc(T** p, size_t count)
{
    const size_t bytes = std::max<size_t>(16, (count * sizeof(T) + 15) & ~size_t(15));
    if (!isg_alloc_allowed(bytes)) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    e = cudaMemset(*p, 0, bytes);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    return e;
}

template <typename T>
void zfree(T*& p)
{
    if (p)
        cudaFree(p);
    p = nullptr;
}

inline int cdiv(long long a, int b) { return int((a + b - 1) / b); }

cudaError_t gemm(ising_mlp_s* m, cudaStream_t st, int rows, int N, int K, const bf16* A, int lda,
                 const bf16* B, int ldb, const float* bias, const bf16* mask, int ldm, int relu, void* C,
                 int ldc, int c_bf16)
{
    TcGemmArgs g{A, B, lda, ldb, rows, N, K, bias, mask, ldm, relu, C, ldc, c_bf16, m->err};
    return launch_tc_gemm(g, st);
}

// bf16 weight copies used by the GEMMs (plain and transposed)
cudaError_t refresh_bf16(ising_mlp_s* m, cudaStream_t st)
{
    to_bf16_kernel<<<cdiv(kW1, 256), 256, 0, st>>>(m->W1(), kHid, kIn, m->W1b, kIn, 0);
    to_bf16_kernel<<<cdiv(kW2, 256), 256, 0, st>>>(m->W2(), kHid, kHid, m->W2b, kHid, 0);
    to_bf16_kernel<<<cdiv(kW2, 256), 256, 0, st>>>(m->W2(), kHid, kHid, m->W2tb, kHid, 1);
    to_bf16_kernel<<<cdiv(kW3, 256), 256, 0, st>>>(m->W3(), kOut, kHid, m->W3b, kHid, 0);
    to_bf16_kernel<<<cdiv(kW3, 256), 256, 0, st>>>(m->W3(), kOut, kHid, m->W3tb, kIn, 1);
    to_bf16_kernel<<<cdiv(kW3, 256), 256, 0, st>>>(m->W3(), kOut, kHid, m->W3tb + kOut, kIn, 1);
    tile_bf16_kernel<<<cdiv(kW1, 256), 256, 0, st>>>(m->W1(), kHid, kIn, m->W1t);
    tile_bf16_kernel<<<cdiv(kW2, 256), 256, 0, st>>>(m->W2(), kHid, kHid, m->W2t);
    tile_bf16_kernel<<<cdiv(kW3, 256), 256, 0, st>>>(m->W3(), kOut, kHid, m->W3t);
    return cudaGetLastError();
}

// L [rows][32] = W3 relu(W2 relu(W1 x + b1) + b2) + b3 for X [rows][64]
cudaError_t forward(ising_mlp_s* m, cudaStream_t st, int rows, const bf16* X, bf16* H1, bf16* H2, float* L)
{
    cudaError_t e = gemm(m, st, rows, kHid, kIn, X, kIn, m->W1b, kIn, m->b1(), nullptr, 0, 1, H1, kHid, 1);
    if (e == cudaSuccess)
        e = gemm(m, st, rows, kHid, kHid, H1, kHid, m->W2b, kHid, m->b2(), nullptr, 0, 1, H2, kHid, 1);
    if (e == cudaSuccess)
        e = gemm(m, st, rows, kOut, kHid, H2, kHid, m->W3b, kHid, m->b3(), nullptr, 0, 0, L, kOut, 0);
    return e;
}

// logits of `rows` (a multiple of 128) tiled input rows by the fused kernel
cudaError_t forward_fused(ising_mlp_s* m, cudaStream_t st, int rows, const void* Xt, float* L)
{
    MlpFusedArgs f{Xt, m->W1t, m->W2t, m->W3t, m->b1(), m->b2(), m->b3(), L, rows / 128, m->err};
    return launch_mlp_fused(f, isg_num_sms(), st);
}

void transpose(const bf16* src, int rows, int cols, int lds, bf16* dst, int ldd, cudaStream_t st)
{
    transpose_kernel<<<dim3(cdiv(cols, 32), cdiv(rows, 32)), dim3(32, 8), 0, st>>>(src, rows, cols, lds, dst, ldd);
}

// Loss and gradients of the batch in Xb / Yb (B rows, B % 128 == 0)
cudaError_t backward(ising_mlp_s* m, cudaStream_t st, int B)
{
    cudaError_t e = forward(m, st, B, m->Xb, m->H1, m->H2, m->L);
    if (e != cudaSuccess)
        return e;
    bce_kernel<<<cdiv(B, 256), 256, 0, st>>>(m->L, m->Yb, B, m->M, 1.f / float(B), m->dL, m->loss);
    // dH2 = relu'(H2) * (dL W3), dH1 = relu'(H1) * (dH2 W2)
    e = gemm(m, st, B, kHid, kIn, m->dL, kIn, m->W3tb, kIn, nullptr, m->H2, kHid, 0, m->dH2, kHid, 1);
    if (e == cudaSuccess)
        e = gemm(m, st, B, kHid, kHid, m->dH2, kHid, m->W2tb, kHid, nullptr, m->H1, kHid, 0, m->dH1, kHid, 1);
    if (e != cudaSuccess)
        return e;
    transpose(m->Xb, B, kIn, kIn, m->XT, B, st);
    transpose(m->H1, B, kHid, kHid, m->H1T, B, st);
    transpose(m->H2, B, kHid, kHid, m->H2T, B, st);
    transpose(m->dL, B, kIn, kIn, m->dLT, B, st);  // hi rows 0..31, lo rows 32..63; 64..127 stay zero
    transpose(m->dH2, B, kHid, kHid, m->dH2T, B, st);
    transpose(m->dH1, B, kHid, kHid, m->dH1T, B, st);
    // weight gradients: sums over the batch of outer products
    e = gemm(m, st, 128, kHid, B, m->dLT, B, m->H2T, B, nullptr, nullptr, 0, 0, m->gW3(), kHid, 0);
    if (e == cudaSuccess)
        e = gemm(m, st, kHid, kHid, B, m->dH2T, B, m->H1T, B, nullptr, nullptr, 0, 0, m->gW2(), kHid, 0);
    if (e == cudaSuccess)
        e = gemm(m, st, kHid, kIn, B, m->dH1T, B, m->XT, B, nullptr, nullptr, 0, 0, m->gW1(), kIn, 0);
    if (e != cudaSuccess)
        return e;
    colsum_kernel<<<1, kIn, 0, st>>>(m->dL, B, kIn, kIn, m->cs64);
    fold_kernel<<<cdiv(kOut * kHid, 256), 256, 0, st>>>(m->gW3(), m->gb3(), m->cs64);
    colsum_kernel<<<1, kHid, 0, st>>>(m->dH2, B, kHid, kHid, m->gb2());
    colsum_kernel<<<1, kHid, 0, st>>>(m->dH1, B, kHid, kHid, m->gb1());
    return cudaGetLastError();
}

cudaError_t adam_step(ising_mlp_s* m, cudaStream_t st, float lr)
{
    ++m->adam_t;
    const float c1 = float(1.0 / (1.0 - std::pow(0.9, double(m->adam_t))));
    const float c2 = float(1.0 / (1.0 - std::pow(0.999, double(m->adam_t))));
    float* mm = m->mom;
    float* vv = m->mom + kPar;
    const long long off[6] = {0, kW1, kW1 + kHid, kW1 + kHid + kW2, kW1 + 2 * kHid + kW2,
                              kW1 + 2 * kHid + kW2 + kW3};
    const int n[6] = {kW1, kHid, kW2, kHid, kW3, kOut};
    float* g[6] = {m->gW1(), m->gb1(), m->gW2(), m->gb2(), m->gW3(), m->gb3()};
    for (int i = 0; i < 6; ++i)
        adam_kernel<<<cdiv(n[i], 256), 256, 0, st>>>(m->par + off[i], g[i], mm + off[i], vv + off[i], n[i], lr,
                                                      c1, c2);
    return refresh_bf16(m, st);
}

int32_t check_err(ising_mlp_s* m, cudaStream_t st)
{
    int h = 0;
    LCK(cudaMemcpyAsync(&h, m->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    LCK(cudaStreamSynchronize(st));
    if (h) {
        LCK(cudaMemsetAsync(m->err, 0, sizeof(int), st));
        LCK(cudaStreamSynchronize(st));
        return isg_fail(ISING_ERR_TIMEOUT, "tensor-core GEMM: a bounded wait gave up");
    }
    return ISING_OK;
}

cudaError_t ensure_batch(ising_mlp_s* m, int B)
{
    if (B <= m->Bcap)
        return cudaSuccess;
    bf16** bufs[12] = {&m->Xb, &m->H1, &m->H2, &m->dL, &m->dH2, &m->dH1,
                       &m->XT, &m->H1T, &m->H2T, &m->dLT, &m->dH2T, &m->dH1T};
    const size_t width[12] = {kIn, kHid, kHid, kIn, kHid, kHid, kIn, kHid, kHid, 128, kHid, kHid};
    for (int i = 0; i < 12; ++i)
        zfree(*bufs[i]);
    zfree(m->L);
    zfree(m->Yb);
    m->Bcap = 0;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 12 && e == cudaSuccess; ++i)
        e = zalloc(bufs[i], size_t(B) * width[i]);
    if (e == cudaSuccess)
        e = zalloc(&m->L, size_t(B) * kOut);
    if (e == cudaSuccess)
        e = zalloc(&m->Yb, size_t(B));
    if (e == cudaSuccess)
        m->Bcap = B;
    return e;
}

cudaError_t ensure_pass(ising_mlp_s* m, long long rows_pad)
{
    if (rows_pad <= m->Pcap)
        return cudaSuccess;
    zfree(m->PX);
    zfree(m->PL);
    zfree(m->Pphi);
    zfree(m->Pold);
    zfree(m->Pprop);
    zfree(m->Pua);
    zfree(m->Pacc);
    m->Pcap = 0;
    cudaError_t e = zalloc(&m->PX, size_t(rows_pad) * kIn);
    if (e == cudaSuccess)
        e = zalloc(&m->PL, size_t(rows_pad) * kOut);
    if (e == cudaSuccess)
        e = zalloc(&m->Pphi, size_t(rows_pad) * kOut);
    if (e == cudaSuccess)
        e = zalloc(&m->Pold, size_t(rows_pad));
    if (e == cudaSuccess)
        e = zalloc(&m->Pprop, size_t(rows_pad));
    if (e == cudaSuccess)
        e = zalloc(&m->Pua, size_t(rows_pad));
    if (e == cudaSuccess)
        e = zalloc(&m->Pacc, size_t(rows_pad));
    if (e == cudaSuccess)
        m->Pcap = rows_pad;
    return e;
}

// fold finished profiling events into the totals (synchronises on them)
cudaError_t resolve_profile(ising_mlp_s* m)
{
    cudaError_t err = cudaSuccess;
    for (size_t i = 0; i < m->ev_pending.size(); ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(m->ev_pending[i].second);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, m->ev_pending[i].first, m->ev_pending[i].second);
        if (e == cudaSuccess) {
            m->prof_ms += ms;
            ++m->prof_launches;
            m->prof_rows += m->ev_rows[i];
        } else if (err == cudaSuccess) {
            err = e;
        }
        cudaEventDestroy(m->ev_pending[i].first);
        cudaEventDestroy(m->ev_pending[i].second);
    }
    m->ev_pending.clear();
    m->ev_rows.clear();
    return err;
}

void free_mlp(ising_mlp_s* m)
{
    resolve_profile(m);
    bf16** b[] = {&m->W1b, &m->W2b, &m->W3b, &m->W2tb, &m->W3tb, &m->Xd, &m->Xb, &m->H1, &m->H2, &m->dL,
                  &m->dH2, &m->dH1, &m->XT, &m->H1T, &m->H2T, &m->dLT, &m->dH2T, &m->dH1T, &m->PX};
    for (auto p : b)
        zfree(*p);
    zfree(m->W1t);
    zfree(m->W2t);
    zfree(m->W3t);
    zfree(m->par);
    zfree(m->mom);
    zfree(m->grad);
    zfree(m->Yd);
    zfree(m->idx);
    zfree(m->L);
    zfree(m->Yb);
    zfree(m->loss);
    zfree(m->cs64);
    zfree(m->err);
    zfree(m->n_acc);
    zfree(m->PL);
    zfree(m->Pphi);
    zfree(m->Pold);
    zfree(m->Pprop);
    zfree(m->Pua);
    zfree(m->Pacc);
}

}  // namespace
}  // namespace isg

// ================================================================ C ABI
namespace isg {
namespace {

// Greedy colouring of the slice graph in site order: each site takes the
// smallest colour none of its spatial neighbours already holds.
int32_t build_colours(ising_s* g)
{
    if (!g->colour_off.empty())
        return ISING_OK;
    const int S = g->S;
    // spatial neighbours of each site (slice 0 rows hold the spatial edges)
    std::vector<std::vector<int>> nbr(S);
    for (int q = 0; q < S; ++q) {
        for (int e = g->row_ptr[q]; e < g->row_ptr[q + 1]; ++e)
            if (g->col[e] < S && g->col[e] != q)
                nbr[q].push_back(g->col[e]);
        std::sort(nbr[q].begin(), nbr[q].end());
        nbr[q].erase(std::unique(nbr[q].begin(), nbr[q].end()), nbr[q].end());
    }
    // smallest-last order: repeatedly remove a site of least remaining degree
    // (lowest index on ties); greedy colouring in the reverse order uses at
    // most (degeneracy + 1) colours, and fewer classes mean fewer launches
    std::vector<int> deg(S);
    std::set<std::pair<int, int>> heap;
    for (int q = 0; q < S; ++q) {
        deg[q] = int(nbr[q].size());
        heap.insert({deg[q], q});
    }
    std::vector<int> order;
    std::vector<char> gone(S, 0);
    while (!heap.empty()) {
        const int q = heap.begin()->second;
        heap.erase(heap.begin());
        gone[q] = 1;
        order.push_back(q);
        for (int j : nbr[q])
            if (!gone[j]) {
                heap.erase({deg[j], j});
                heap.insert({--deg[j], j});
            }
    }
    std::vector<int> colour(S, -1);
    int ncol = 0;
    std::vector<int> seen;
    for (auto it = order.rbegin(); it != order.rend(); ++it) {
        const int q = *it;
        seen.assign(size_t(ncol) + 1, 0);
        for (int j : nbr[q])
            if (colour[j] >= 0)
                seen[colour[j]] = 1;
        int k = 0;
        while (seen[k])
            ++k;
        colour[q] = k;
        ncol = std::max(ncol, k + 1);
    }
    std::vector<int> sites;
    g->colour_off.assign(1, 0);
    for (int k = 0; k < ncol; ++k) {
        for (int q = 0; q < S; ++q)
            if (colour[q] == k)
                sites.push_back(q);
        g->colour_off.push_back(int(sites.size()));
    }
    std::vector<int> sp_off(1, 0);
    std::vector<int2> sp_nbr;
    long long max_j2 = 0;
    for (int q = 0; q < S; ++q) {
        long long j2 = 0;
        for (int e = g->row_ptr[q]; e < g->row_ptr[q + 1]; ++e)
            if (g->col[e] < S) {
                sp_nbr.push_back(make_int2(g->col[e], g->J[e]));
                j2 += 2LL * std::llabs((long long)g->J[e]);
            }
        max_j2 = std::max(max_j2, j2);
        sp_off.push_back(int(sp_nbr.size()));
    }
    g->sp_simd = max_j2 <= 127 ? 1 : 0;
    cudaError_t e = zalloc(&g->d_colour_sites, sites.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_colour_sites, sites.data(), sites.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = zalloc(&g->d_sp_off, sp_off.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d_sp_off, sp_off.data(), sp_off.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = zalloc(&g->d_sp_nbr, sp_nbr.size());
    if (e == cudaSuccess && !sp_nbr.empty())
        e = cudaMemcpy(g->d_sp_nbr, sp_nbr.data(), sp_nbr.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        zfree(g->d_colour_sites);
        zfree(g->d_sp_off);
        zfree(g->d_sp_nbr);
        g->colour_off.clear();
        return cuda_err(e, "colour classes");
    }
    g->colour_sites = sites;
    return ISING_OK;
}

LearnedArgs learned_args(ising_s* g, ising_mlp_s* m)
{
    LearnedArgs a{};
    a.S = g->S;
    a.M = g->M;
    a.N = g->n;
    a.R = g->R;
    a.row_ptr = g->d_row_ptr;
    a.col = g->d_col;
    a.J = g->d_J;
    a.h = g->d_h;
    a.jtau = g->d_jtau;
    a.pos = g->d_pos;
    a.spins = g->d_spins;
    a.E = g->d_E;
    a.temp_of_slot = g->d_temp;
    a.betas = g->d_betas;
    a.betas32 = g->d_betas32;
    a.sp_off = g->d_sp_off;
    a.sp_nbr = g->d_sp_nbr;
    a.colbits = g->d_colbits;
    a.sp_simd = g->sp_simd;
    a.seed = g->seed;
    a.inst = g->inst;
    a.pass = uint32_t(g->learned_passes);
    a.phi = m->Pphi;
    a.X = m->PX;
    a.L = m->PL;
    a.old_bits = m->Pold;
    a.prop_bits = m->Pprop;
    a.acc_word = m->Pua;
    a.accepted = m->Pacc;
    a.n_acc = m->n_acc;
    a.n_exact = m->n_acc + 1;
    a.fields = g->d_fields;
    a.field_bits = g->field_bits;
    a.n_changed = m->n_acc + 2;
    return a;
}

}  // namespace
}  // namespace isg

using namespace isg;

extern "C" {

int32_t ising_mlp_create(int32_t n_slices, uint32_t seed, int64_t capacity, ising_mlp_t* out)
{
    if (!out)
        return isg_fail(ISING_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_slices < 1 || n_slices > kOut)
        return isg_fail(ISING_ERR_INVALID_ARG, "n_slices must be in 1..32");
    if (capacity < 0 || capacity > (1LL << 31) - 1)
        return isg_fail(ISING_ERR_INVALID_ARG, "capacity must be in 0..2^31-1");
    int32_t rc = isg_device_setup();
    if (rc)
        return rc;
    auto* m = new ising_mlp_s();
    m->M = n_slices;
    m->seed = seed;
    m->cap = capacity;
    cudaError_t e = zalloc(&m->par, kPar);
    if (e == cudaSuccess)
        e = zalloc(&m->mom, 2 * size_t(kPar));
    if (e == cudaSuccess)
        e = zalloc(&m->grad, kGrad);
    if (e == cudaSuccess)
        e = zalloc(&m->W1b, kW1);
    if (e == cudaSuccess)
        e = zalloc(&m->W2b, kW2);
    if (e == cudaSuccess)
        e = zalloc(&m->W2tb, kW2);
    if (e == cudaSuccess)
        e = zalloc(&m->W3b, kW3);
    if (e == cudaSuccess)
        e = zalloc(&m->W3tb, size_t(kHid) * kIn);
    if (e == cudaSuccess)
        e = zalloc(&m->W1t, size_t(kW1) * 2);
    if (e == cudaSuccess)
        e = zalloc(&m->W2t, size_t(kW2) * 2);
    if (e == cudaSuccess)
        e = zalloc(&m->W3t, size_t(kW3) * 2);
    if (e == cudaSuccess)
        e = zalloc(&m->Xd, size_t(std::max<int64_t>(capacity, 1)) * kIn);
    if (e == cudaSuccess)
        e = zalloc(&m->Yd, size_t(std::max<int64_t>(capacity, 1)));
    if (e == cudaSuccess)
        e = zalloc(&m->idx, size_t(std::max<int64_t>(capacity, 1)));
    if (e == cudaSuccess)
        e = zalloc(&m->loss, 1);
    if (e == cudaSuccess)
        e = zalloc(&m->cs64, kIn);
    if (e == cudaSuccess)
        e = zalloc(&m->err, 1);
    if (e == cudaSuccess)
        e = zalloc(&m->n_acc, 3);
    if (e != cudaSuccess) {
        free_mlp(m);
        delete m;
        return cuda_err(e, "ising_mlp_create");
    }
    // uniform on +-1/sqrt(fan_in), biases 0, padding 0
    std::vector<float> p(kPar, 0.f);
    std::mt19937 gen(seed);
    auto fill = [&](float* w, int rows, int cols, int ld, int fan_in) {
        const float a = 1.f / std::sqrt(float(fan_in));
        std::uniform_real_distribution<float> u(-a, a);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c)
                w[size_t(r) * ld + c] = u(gen);
    };
    fill(p.data(), kHid, n_slices + 1, kIn, n_slices + 1);
    fill(p.data() + kW1 + kHid, kHid, kHid, kHid, kHid);
    fill(p.data() + kW1 + 2 * kHid + kW2, n_slices, kHid, kHid, kHid);
    e = cudaMemcpy(m->par, p.data(), sizeof(float) * kPar, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = refresh_bf16(m, nullptr);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_mlp(m);
        delete m;
        return cuda_err(e, "ising_mlp_create");
    }
    *out = m;
    return ISING_OK;
}

int32_t ising_mlp_set_stream(ising_mlp_t m, void* cuda_stream)
{
    if (!m)
        return isg_fail(ISING_ERR_INVALID_ARG, "network is NULL");
    m->stream = static_cast<cudaStream_t>(cuda_stream);
    return ISING_OK;
}

int64_t ising_mlp_n_params(ising_mlp_t m)
{
    if (!m)
        return 0;
    const int M = m->M;
    return int64_t(kHid) * (M + 1) + kHid + kW2 + kHid + int64_t(M) * kHid + M;
}

int32_t ising_mlp_get_params(ising_mlp_t m, float* out)
{
    if (!m || !out)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument");
    std::vector<float> p(kPar);
    LCK(cudaStreamSynchronize(m->stream));
    LCK(cudaMemcpy(p.data(), m->par, sizeof(float) * kPar, cudaMemcpyDeviceToHost));
    const int M = m->M;
    float* o = out;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c <= M; ++c)
            *o++ = p[size_t(r) * kIn + c];
    o = std::copy(p.begin() + kW1, p.begin() + kW1 + kHid + kW2 + kHid, o);
    const size_t w3 = kW1 + 2 * kHid + kW2;
    o = std::copy(p.begin() + w3, p.begin() + w3 + size_t(M) * kHid, o);
    std::copy(p.begin() + w3 + kW3, p.begin() + w3 + kW3 + M, o);
    return ISING_OK;
}

int32_t ising_mlp_set_params(ising_mlp_t m, const float* in)
{
    if (!m || !in)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument");
    std::vector<float> p(kPar, 0.f);
    const int M = m->M;
    const float* s = in;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c <= M; ++c)
            p[size_t(r) * kIn + c] = *s++;
    std::copy(s, s + kHid + kW2 + kHid, p.begin() + kW1);
    s += kHid + kW2 + kHid;
    const size_t w3 = kW1 + 2 * kHid + kW2;
    std::copy(s, s + size_t(M) * kHid, p.begin() + w3);
    s += size_t(M) * kHid;
    std::copy(s, s + M, p.begin() + w3 + kW3);
    LCK(cudaStreamSynchronize(m->stream));
    LCK(cudaMemcpy(m->par, p.data(), sizeof(float) * kPar, cudaMemcpyHostToDevice));
    LCK(cudaMemset(m->mom, 0, sizeof(float) * 2 * kPar));
    m->adam_t = 0;
    LCK(refresh_bf16(m, m->stream));
    LCK(cudaStreamSynchronize(m->stream));
    return ISING_OK;
}

}  // extern "C"

namespace isg {
namespace {

std::vector<bf16> pack_inputs(const float* X, int B, int M)
{
    std::vector<bf16> x(size_t(B) * kIn, __float2bfloat16(0.f));
    for (int b = 0; b < B; ++b)
        for (int c = 0; c <= M; ++c)
            x[size_t(b) * kIn + c] = __float2bfloat16(X[size_t(b) * (M + 1) + c]);
    return x;
}

}  // namespace
}  // namespace isg

extern "C" {

int32_t ising_mlp_forward(ising_mlp_t m, int32_t B, const float* X, float* L)
{
    if (!m || !X || !L || B < 1)
        return isg_fail(ISING_ERR_INVALID_ARG, "forward: NULL argument or B < 1");
    const int rows_pad = cdiv(B, 128) * 128;
    cudaStream_t st = m->stream;
    LCK(cudaStreamSynchronize(st));
    LCK(ensure_pass(m, rows_pad));
    const std::vector<bf16> x = pack_inputs(X, B, m->M);
    std::vector<unsigned char> xt(size_t(rows_pad) * kIn * 2, 0);
    for (int b = 0; b < B; ++b)
        for (int c = 0; c < kIn; ++c)
            std::memcpy(xt.data() + size_t(b >> 7) * 16384 + tiled_offset(128, b & 127, c), &x[size_t(b) * kIn + c], 2);
    LCK(cudaMemcpyAsync(m->PX, xt.data(), xt.size(), cudaMemcpyHostToDevice, st));
    LCK(forward_fused(m, st, rows_pad, m->PX, m->PL));
    std::vector<float> l(size_t(rows_pad) * kOut);  // tiles stored column by column
    LCK(cudaMemcpyAsync(l.data(), m->PL, sizeof(float) * l.size(), cudaMemcpyDeviceToHost, st));
    int32_t rc = check_err(m, st);
    if (rc)
        return rc;
    for (int b = 0; b < B; ++b)
        for (int t = 0; t < m->M; ++t)
            L[size_t(b) * m->M + t] = l[size_t(b >> 7) * (128 * kOut) + size_t(t) * 128 + (b & 127)];
    return ISING_OK;
}

int32_t ising_mlp_grad(ising_mlp_t m, int32_t B, const float* X, const uint32_t* Y, float* grad, float* loss)
{
    if (!m || !X || !Y || !grad || B < 128 || B % 128)
        return isg_fail(ISING_ERR_INVALID_ARG, "grad: NULL argument or B not a positive multiple of 128");
    cudaStream_t st = m->stream;
    LCK(cudaStreamSynchronize(st));
    LCK(ensure_batch(m, B));
    const std::vector<bf16> x = pack_inputs(X, B, m->M);
    LCK(cudaMemcpyAsync(m->Xb, x.data(), sizeof(bf16) * x.size(), cudaMemcpyHostToDevice, st));
    LCK(cudaMemcpyAsync(m->Yb, Y, sizeof(uint32_t) * B, cudaMemcpyHostToDevice, st));
    LCK(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
    LCK(backward(m, st, B));
    std::vector<float> g(kGrad);
    float lsum = 0.f;
    LCK(cudaMemcpyAsync(g.data(), m->grad, sizeof(float) * kGrad, cudaMemcpyDeviceToHost, st));
    LCK(cudaMemcpyAsync(&lsum, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
    int32_t rc = check_err(m, st);
    if (rc)
        return rc;
    const int M = m->M;
    float* o = grad;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c <= M; ++c)
            *o++ = g[size_t(r) * kIn + c];
    o = std::copy(g.begin() + kW1, g.begin() + kW1 + kHid + kW2 + kHid, o);
    const size_t w3 = kW1 + 2 * kHid + kW2;
    o = std::copy(g.begin() + w3, g.begin() + w3 + size_t(M) * kHid, o);
    std::copy(g.begin() + w3 + kGW3, g.begin() + w3 + kGW3 + M, o);
    if (loss)
        *loss = lsum / float(B);
    return ISING_OK;
}

int32_t ising_mlp_collect(ising_mlp_t m, ising_t h) { return ising_mlp_collect_flags(m, h, 0u); }

int32_t ising_mlp_collect_flags(ising_mlp_t m, ising_t h, uint32_t flags)
{
    if (flags & ~uint32_t(ISING_COLLECT_ORIENTED))
        return isg_fail(ISING_ERR_INVALID_ARG, "unknown collect flags");
    if (!m || !h)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!h->inited)
        return isg_fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (h->split)
        return isg_fail(ISING_ERR_UNSUPPORTED, "learned column moves use the plain Trotter coupling, not split couplings");
    if (h->M != m->M)
        return isg_fail(ISING_ERR_INVALID_ARG, "the handle's slice count differs from the network's");
    const long long rows = (long long)h->R * h->S;
    if (m->n_rec + rows > m->cap)
        return isg_fail(ISING_ERR_INVALID_ARG, "record capacity exceeded");
    LearnedArgs a = learned_args(h, m);
    collect_kernel<<<cdiv(rows, 256), 256, 0, h->stream>>>(a, m->Xd + size_t(m->n_rec) * kIn, m->Yd + m->n_rec,
                                                           (flags & ISING_COLLECT_ORIENTED) ? 1 : 0);
    LCK(cudaGetLastError());
    LCK(cudaStreamSynchronize(h->stream));
    m->n_rec += rows;
    return ISING_OK;
}

int64_t ising_mlp_n_records(ising_mlp_t m) { return m ? m->n_rec : 0; }

int32_t ising_mlp_clear_records(ising_mlp_t m)
{
    if (!m)
        return isg_fail(ISING_ERR_INVALID_ARG, "network is NULL");
    m->n_rec = 0;
    return ISING_OK;
}

int32_t ising_mlp_get_records(ising_mlp_t m, int64_t start, int64_t n, float* X, uint32_t* Y)
{
    if (!m || n < 0 || start < 0 || (n > 0 && (!X || !Y)))
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument or negative range");
    if (start + n > m->n_rec)
        return isg_fail(ISING_ERR_INVALID_ARG, "range beyond the recorded rows");
    if (n == 0)
        return ISING_OK;
    std::vector<bf16> xb(size_t(n) * kIn);
    LCK(cudaMemcpy(xb.data(), m->Xd + size_t(start) * kIn, xb.size() * sizeof(bf16), cudaMemcpyDeviceToHost));
    LCK(cudaMemcpy(Y, m->Yd + start, size_t(n) * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c <= m->M; ++c)
            X[i * (m->M + 1) + c] = __bfloat162float(xb[size_t(i) * kIn + c]);
    return ISING_OK;
}

int32_t ising_mlp_train(ising_mlp_t m, int32_t epochs, int32_t batch, float lr, float* loss)
{
    if (!m || epochs < 0 || batch < 128 || batch % 128 || !(lr > 0.f))
        return isg_fail(ISING_ERR_INVALID_ARG, "train: epochs >= 0, batch a positive multiple of 128, lr > 0");
    const long long nb = m->n_rec / batch;
    if (nb < 1)
        return isg_fail(ISING_ERR_INVALID_ARG, "train: fewer records than one batch");
    cudaStream_t st = m->stream;
    LCK(cudaStreamSynchronize(st));
    LCK(ensure_batch(m, batch));
    std::vector<int> order(size_t(m->n_rec));
    float last = 0.f;
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long i = 0; i < m->n_rec; ++i)
            order[size_t(i)] = int(i);
        std::mt19937_64 gen(uint64_t(m->seed) + uint64_t(ep));
        std::shuffle(order.begin(), order.end(), gen);
        LCK(cudaMemcpyAsync(m->idx, order.data(), sizeof(int) * order.size(), cudaMemcpyHostToDevice, st));
        LCK(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
        for (long long b = 0; b < nb; ++b) {
            gather_batch_kernel<<<cdiv(batch * (kIn / 8), 256), 256, 0, st>>>(m->Xd, m->Yd, m->idx + b * batch,
                                                                              batch, m->Xb, m->Yb);
            LCK(backward(m, st, batch));
            LCK(adam_step(m, st, lr));
        }
        float lsum = 0.f;
        LCK(cudaMemcpyAsync(&lsum, m->loss, sizeof(float), cudaMemcpyDeviceToHost, st));
        int32_t rc = check_err(m, st);
        if (rc)
            return rc;
        last = lsum / float(nb * batch);
    }
    if (loss)
        *loss = last;
    return ISING_OK;
}

int32_t ising_learned_pass(ising_t h, ising_mlp_t m, uint32_t flags, ising_learned_stats_t* stats,
                           const ising_learned_trace_t* trace)
{
    if (!m || !h)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!h->inited)
        return isg_fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (h->split)
        return isg_fail(ISING_ERR_UNSUPPORTED, "learned column moves use the plain Trotter coupling, not split couplings");
    if (h->M != m->M)
        return isg_fail(ISING_ERR_INVALID_ARG, "the handle's slice count differs from the network's");
    const long long total = (long long)h->R * h->S;
    if (total > (1LL << 31) - 256)
        return isg_fail(ISING_ERR_UNSUPPORTED, "learned passes need R * S below 2^31");
    if (trace && trace->capacity < total)
        return isg_fail(ISING_ERR_INVALID_ARG, "trace capacity below R * S rows");
    int32_t rc = build_colours(h);
    if (rc)
        return rc;
    // column bits of the replicas (their lifetime: ising_replicas_init frees them)
    if (h->colbits_cap < size_t(total)) {
        zfree(h->d_colbits);
        h->colbits_cap = 0;
        LCK(zalloc(&h->d_colbits, size_t(total)));
        h->colbits_cap = size_t(total);
    }
    cudaStream_t st = h->stream;
    long long maxrows = 0;
    for (size_t c = 0; c + 1 < h->colour_off.size(); ++c)
        maxrows = std::max(maxrows, (long long)h->R * (h->colour_off[c + 1] - h->colour_off[c]));
    const long long maxpad = (maxrows + 127) / 128 * 128;
    if (maxpad > (1LL << 31) - 1)
        return isg_fail(ISING_ERR_UNSUPPORTED, "a colour class holds more than 2^31 rows");
    if (maxpad > m->Pcap) {  // growing the workspace needs the network idle
        LCK(cudaStreamSynchronize(m->stream));
        LCK(cudaStreamSynchronize(st));
        LCK(ensure_pass(m, maxpad));
    }
    LCK(cudaMemsetAsync(m->n_acc, 0, 3 * sizeof(unsigned long long), st));
    {
        const LearnedArgs a = learned_args(h, m);
        learned_colbits_kernel<<<cdiv(total, 256), 256, 0, st>>>(a);
    }
    long long done = 0;
    for (size_t c = 0; c + 1 < h->colour_off.size(); ++c) {
        const int ncols = h->colour_off[c + 1] - h->colour_off[c];
        const int rows = h->R * ncols;
        const int rows_pad = cdiv(rows, 128) * 128;
        LearnedArgs a = learned_args(h, m);
        a.ncols = ncols;
        a.rows = rows;
        a.sites = h->d_colour_sites + h->colour_off[c];
        a.fp64_only = (flags & ISING_LEARNED_FP64_ONLY) ? 1 : 0;
        a.mixture = (flags & ISING_LEARNED_MIXTURE) ? 1 : 0;
        learned_gather_kernel<<<cdiv(rows_pad, 128), 128, 0, st>>>(a, rows_pad);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (m->profiling) {
            LCK(cudaEventCreate(&e0));
            LCK(cudaEventCreate(&e1));
            LCK(cudaEventRecord(e0, st));
        }
        LCK(forward_fused(m, st, rows_pad, m->PX, m->PL));
        if (m->profiling) {
            LCK(cudaEventRecord(e1, st));
            m->ev_pending.emplace_back(e0, e1);
            m->ev_rows.push_back(rows);
        }
        learned_mh_kernel<<<cdiv(rows, kMhRows), kMhThreads, 0, st>>>(a);
        LCK(cudaGetLastError());
        if (trace) {
            auto d2h = [&](void* dst, const void* src, size_t bytes) {
                return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, st) : cudaSuccess;
            };
            LCK(d2h(trace->phi ? trace->phi + done * kOut : nullptr, m->Pphi, sizeof(int) * size_t(rows) * kOut));
            std::vector<float> lt;  // logits, tiles stored column by column
            if (trace->logits) {
                lt.resize(size_t(rows_pad) * kOut);
                LCK(cudaMemcpyAsync(lt.data(), m->PL, sizeof(float) * lt.size(), cudaMemcpyDeviceToHost, st));
            }
            LCK(d2h(trace->old_bits ? trace->old_bits + done : nullptr, m->Pold, sizeof(uint32_t) * rows));
            LCK(d2h(trace->prop_bits ? trace->prop_bits + done : nullptr, m->Pprop, sizeof(uint32_t) * rows));
            LCK(d2h(trace->accepted ? trace->accepted + done : nullptr, m->Pacc, size_t(rows)));
            LCK(cudaStreamSynchronize(st));
            if (trace->logits)
                for (int i = 0; i < rows; ++i)
                    for (int t = 0; t < kOut; ++t)
                        trace->logits[(done + i) * kOut + t] =
                            lt[size_t(i >> 7) * (128 * kOut) + size_t(t) * 128 + (i & 127)];
            for (int i = 0; i < rows; ++i) {
                const int r = i / ncols;
                if (trace->replica)
                    trace->replica[done + i] = r;
                if (trace->site)
                    trace->site[done + i] = h->colour_sites[h->colour_off[c] + i - r * ncols];
            }
        }
        done += rows;
    }
    {
        const LearnedArgs a = learned_args(h, m);
        if (h->field_bits == 16)
            learned_fields_kernel<int16_t><<<cdiv(total, 256), 256, 0, st>>>(a);
        else
            learned_fields_kernel<int><<<cdiv(total, 256), 256, 0, st>>>(a);
        LCK(cudaGetLastError());
    }
    ++h->learned_passes;
    if (!stats && !trace)
        return ISING_OK;  // asynchronous: errors surface at the next synchronising call
    unsigned long long acc[3] = {0, 0, 0};
    LCK(cudaMemcpyAsync(acc, m->n_acc, sizeof(acc), cudaMemcpyDeviceToHost, st));
    rc = check_err(m, st);
    if (rc)
        return rc;
    if (stats) {
        stats->proposed = uint64_t(total);
        stats->accepted = acc[0];
        stats->exact_decisions = acc[1];
        stats->changed = acc[2];
    }
    return ISING_OK;
}

int32_t ising_mlp_set_profiling(ising_mlp_t m, int32_t on)
{
    if (!m)
        return isg_fail(ISING_ERR_INVALID_ARG, "network is NULL");
    m->profiling = on != 0;
    return ISING_OK;
}

int32_t ising_mlp_get_stats(ising_mlp_t m, ising_mlp_stats_t* out)
{
    if (!m || !out)
        return isg_fail(ISING_ERR_INVALID_ARG, "NULL argument");
    LCK(resolve_profile(m));
    out->network_launches = m->prof_launches;
    out->network_rows = m->prof_rows;
    out->network_ms = m->prof_ms;
    return ISING_OK;
}

int32_t ising_mlp_destroy(ising_mlp_t m)
{
    if (!m)
        return ISING_OK;
    cudaStreamSynchronize(m->stream);
    free_mlp(m);
    delete m;
    return ISING_OK;
}

}  // extern "C"
