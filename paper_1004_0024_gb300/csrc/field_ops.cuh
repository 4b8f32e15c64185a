// Shared-memory field storage and the Trotter part of the local field,
// used by both sweep kernels.
#pragma once
#include <cstdint>

namespace isg {

__host__ __device__ inline uint32_t r16(uint32_t x) { return (x + 15u) & ~15u; }

template <typename FT>
struct Fsp;

template <>
struct Fsp<int32_t> {
    static constexpr int kBytes = 4;
    __device__ static int ld(const void* b, int i) { return static_cast<const int*>(b)[i]; }
    __device__ static void st(void* b, int i, int v) { static_cast<int*>(b)[i] = v; }
    __device__ static void add(void* b, int i, int d) { atomicAdd(static_cast<int*>(b) + i, d); }
};

// int16 fields are stored biased (f + 32768) as the halves of 32-bit words.
// A value bounded by |f| <= 32767 keeps each biased half inside [1, 65535],
// so adding a delta to the containing word never carries into the other half
// and a 32-bit atomic add updates one int16 field exactly.
template <>
struct Fsp<int16_t> {
    static constexpr int kBytes = 2;
    __device__ static int ld(const void* b, int i)
    {
        return int(static_cast<const uint16_t*>(b)[i]) - 32768;
    }
    __device__ static void st(void* b, int i, int v)
    {
        static_cast<uint16_t*>(b)[i] = static_cast<uint16_t>(v + 32768);
    }
    __device__ static void add(void* b, int i, int d)
    {
        atomicAdd(static_cast<unsigned*>(b) + (i >> 1), static_cast<unsigned>(d) << ((i & 1) << 4));
    }
};

// Trotter part of the field of spin (column cb, slice t): Jtau * (s_{t-1} +
// s_{t+1}) on a ring of M >= 3 slices, Jtau * s_other for M = 2, 0 for M = 1.
__device__ __forceinline__ int trotter_field(const uint32_t* cb, int t, int M, int jt)
{
    if (M >= 3) {
        const int tm = (t == 0) ? M - 1 : t - 1;
        const int tp = (t == M - 1) ? 0 : t + 1;
        const int bm = (cb[tm >> 5] >> (tm & 31)) & 1;
        const int bp = (cb[tp >> 5] >> (tp & 31)) & 1;
        return jt * (2 * (bm + bp) - 2);
    }
    if (M == 2) {
        const int o = 1 - t;
        return jt * (2 * int((cb[0] >> o) & 1u) - 1);
    }
    return 0;
}

constexpr long long kWaitPolls = 1LL << 22;

}  // namespace isg
