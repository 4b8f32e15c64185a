// Host side of the C ABI declared in include/ising_gb300.h.
//
// ising_create validates the CSR model, verifies the declared slice
// structure, computes the slice wavefront levels and packs the per-slice
// tables.  ising_replicas_init builds the FP64 flip and swap thresholds and
// draws the initial replicas.  ising_sweep / ising_pt_swap / ising_run plan a
// sequence of launches (MT19937 word generation, wavefront sweeps, PT passes)
// that reads every mutable quantity from device memory, so a recorded CUDA
// graph can be replayed any number of times.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <utility>
#include <tuple>
#include <vector>

#include "host_pool.h"
#include "ising_gb300.h"
#include "ising_internal.cuh"
#include "split_math.cuh"

using namespace isg;

namespace {

thread_local std::string g_err = "";

int32_t fail(int32_t code, const std::string& msg)
{
    g_err = msg;
    return code;
}

int32_t cuda_fail(cudaError_t e, const char* what)
{
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? ISING_ERR_OOM : ISING_ERR_CUDA;
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess)                     \
            return cuda_fail(e_, #call);           \
    } while (0)

// Process-wide cap on one device allocation (ising_set_alloc_cap; 0 = none):
// an out-of-memory stand-in for tests of the error paths.
std::atomic<unsigned long long> g_alloc_cap{0};

bool alloc_allowed(size_t bytes)
{
    const unsigned long long cap = g_alloc_cap.load();
    return cap == 0 || bytes <= cap;
}

template <typename T>
int32_t dalloc(T** p, size_t count)
{
    size_t bytes = ((count * sizeof(T)) + 15) & ~size_t(15);
    if (bytes == 0)
        bytes = 16;
    if (!alloc_allowed(bytes)) {
        *p = nullptr;
        return fail(ISING_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap");
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    e = cudaMemset(*p, 0, bytes);
    if (e == cudaSuccess)  // allocations are rare: finish the fill before any stream uses it
        e = cudaStreamSynchronize(0);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemset");
    return ISING_OK;
}

template <typename T>
void dfree(T*& p)
{
    if (p)
        cudaFree(p);
    p = nullptr;
}

// Large blocks (the MT19937 word buffers, gigabytes) are not returned to the
// driver when a handle lets them go: freeing and re-mapping them costs
// milliseconds per handle.  Up to kBigKeep freed blocks wait here, after a
// device synchronisation (so no kernel of the old owner still touches them),
// for an allocation of at most their size that needs no more than 5/4 of
// it; ising_release_cached_memory frees them, and so does an allocation
// that fails.  Their contents are undefined (no zero fill).
constexpr size_t kBigBlock = size_t(256) << 20;
constexpr size_t kBigKeep = 2;
std::mutex g_big_mu;
std::multimap<size_t, void*> g_big_free;       // size -> block
std::unordered_map<void*, size_t> g_big_live;  // block -> size

void big_release_all()
{
    std::lock_guard<std::mutex> lk(g_big_mu);
    for (auto& kv : g_big_free)
        cudaFree(kv.second);
    g_big_free.clear();
}

template <typename T>
int32_t big_alloc(T** p, size_t count)
{
    const size_t bytes = std::max<size_t>(16, ((count * sizeof(T)) + 15) & ~size_t(15));
    *p = nullptr;
    if (!alloc_allowed(bytes))
        return fail(ISING_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap");
    if (bytes >= kBigBlock) {
        std::lock_guard<std::mutex> lk(g_big_mu);
        auto it = g_big_free.lower_bound(bytes);
        if (it != g_big_free.end() && it->first - bytes <= bytes / 4) {
            *p = static_cast<T*>(it->second);
            g_big_live[it->second] = it->first;
            g_big_free.erase(it);
            return ISING_OK;
        }
    }
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    if (e == cudaErrorMemoryAllocation) {  // give the cached blocks back and retry once
        cudaGetLastError();
        big_release_all();
        e = cudaMalloc(reinterpret_cast<void**>(p), bytes);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    if (bytes >= kBigBlock) {
        std::lock_guard<std::mutex> lk(g_big_mu);
        g_big_live[*p] = bytes;
    }
    return ISING_OK;
}

template <typename T>
void big_free(T*& p)
{
    if (!p)
        return;
    void* v = p;
    p = nullptr;
    std::lock_guard<std::mutex> lk(g_big_mu);
    auto it = g_big_live.find(v);
    if (it == g_big_live.end()) {
        cudaFree(v);
        return;
    }
    const size_t bytes = it->second;
    g_big_live.erase(it);
    if (g_big_free.size() < kBigKeep && cudaDeviceSynchronize() == cudaSuccess) {
        g_big_free.emplace(bytes, v);
        return;
    }
    cudaFree(v);
}

template <typename T>
int32_t upload(T** d, const std::vector<T>& h)
{
    // no fill of what the copy overwrites: only the 16-byte rounding tail is
    // zeroed; the synchronous copy on the legacy stream follows the fill, so
    // both are complete on return
    size_t bytes = ((h.size() * sizeof(T)) + 15) & ~size_t(15);
    if (bytes == 0)
        bytes = 16;
    *d = nullptr;
    if (!alloc_allowed(bytes))
        return fail(ISING_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes exceeds the cap");
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(d), bytes);
    if (e != cudaSuccess) {
        *d = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    const size_t data = h.size() * sizeof(T);
    if (bytes > data)
        CK(cudaMemset(reinterpret_cast<unsigned char*>(*d) + data, 0, bytes - data));
    if (!h.empty())
        CK(cudaMemcpy(*d, h.data(), data, cudaMemcpyHostToDevice));
    return ISING_OK;
}

int g_num_sms = 0;
int g_coop = 0;
std::once_flag g_once;
cudaError_t g_init_err = cudaSuccess;

cudaError_t device_setup()
{
    std::call_once(g_once, [] {
        int dev = 0;
        g_init_err = cudaGetDevice(&dev);
        if (g_init_err == cudaSuccess)
            g_init_err = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_init_err == cudaSuccess)
            g_init_err = sweep_set_smem_limits();
        if (g_init_err == cudaSuccess)
            g_init_err = fast_set_smem_limits();
        if (g_init_err == cudaSuccess)
            g_init_err = mt_gen_set_smem_limit();
        if (g_init_err == cudaSuccess)
            g_init_err = tc_gemm_setup();
        if (g_init_err == cudaSuccess)
            g_init_err = mlp_fused_setup();
        int coop = 0;
        if (g_init_err == cudaSuccess)
            g_init_err = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        g_coop = coop;
    });
    return g_init_err;
}

// MT19937 init_genrand (Matsumoto & Nishimura): x_0 = seed,
// x_i = 1812433253 (x_{i-1} ^ (x_{i-1} >> 30)) + i.
void mt_seed_ring(uint32_t seed, uint32_t* ring)
{
    ring[0] = seed;
    for (int i = 1; i < 624; ++i)
        ring[i] = 1812433253u * (ring[i - 1] ^ (ring[i - 1] >> 30)) + uint32_t(i);
    for (int i = 624; i < kMtRing; ++i)
        ring[i] = 0u;
}

}  // namespace

#include "handle.h"
#include "packed_impl.cuh"


void ising_s::drop_graphs()
{
    for (auto& kv : graphs)
        cudaGraphExecDestroy(kv.second);
    graphs.clear();
}

void ising_s::free_replicas()
{
    dfree(d_obs);
    dfree(d_widen);
    widen_cap = 0;
    dfree(d_colbits);  // sized for these replicas (learned passes)
    colbits_cap = 0;
    drop_graphs();
    dfree(d_spins);
    if (d_fields)
        cudaFree(d_fields);
    d_fields = nullptr;
    dfree(d_E);
    dfree(d_temp);
    dfree(d_slot);
    dfree(d_err);
    dfree(d_swap_acc);
    dfree(d_counters);
    dfree(d_mtpos);
    dfree(d_done);
    dfree(d_thr);
    dfree(d_swthr);
    dfree(d_mtring);
    dfree(d_swoff);
    dfree(d_swlen);
    dfree(d_betas);
    dfree(d_betas32);
    big_free(d_wbuf);
    dfree(d_swbuf);
    dfree(d_Epub);
    dfree(d_gridbar);
    dfree(d_C);
    dfree(d_Cpub);
    dfree(d_dbeta);
    dfree(d_dK);
    split = false;
    split_ks = 0;
    trotter_K.clear();
    wbuf_cap = swbuf_cap = 0;
    inited = false;
}

void ising_s::free_all()
{
    free_replicas();
    for (auto& ev : ev_pending) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    ev_pending.clear();
    if (cap_stream)
        cudaStreamDestroy(cap_stream);
    cap_stream = nullptr;
    dfree(d_row_ptr);
    dfree(d_col);
    dfree(d_J);
    dfree(d_h);
    dfree(d_nbr_off);
    dfree(d_jtau);
    dfree(d_lev0);
    dfree(d_site);
    dfree(d_pos);
    dfree(d_nbr);
    dfree(d_colour_sites);
    dfree(d_track_off);
    dfree(d_track_col);
    dfree(d_pk);
    dfree(d_sp_off);
    dfree(d_sp_nbr);
    dfree(d_colbits);
    colour_off.clear();
    colour_sites.clear();
}

namespace {

// ---------------------------------------------------------- validation
// Also returns, for a valid model, kmax = max_i |h_i| + sum_j |J_ij| and
// ebound = sum_i |h_i| + sum over pairs of |J_ij| (computed in the same pass).
int32_t validate_csr(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* J,
                     const int32_t* h, long long* kmax, long long* ebound)
{
    if (row_ptr[0] != 0)
        return fail(ISING_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (int i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i])
            return fail(ISING_ERR_INVALID_ARG, "row_ptr must be non-decreasing");
    // every row's (column, J) entries sorted in one flat array; rows are
    // checked in parallel chunks, and of each phase the error of the lowest
    // row is reported (the one a row-by-row pass would meet first)
    const long long nnz = row_ptr[n];
    std::vector<std::pair<int, int>> ent_mem(size_t(std::max<long long>(nnz, 1)));
    std::pair<int, int>* const ent = ent_mem.data();
    struct RowErr {
        int row = INT32_MAX, code = ISING_OK;
        std::string msg;
    };
    const int nthr = n >= 8192 ? host_threads() : 1;
    // per-thread partial sums, one cache line each
    struct alignas(64) Part {
        long long km = 0, eb = 0, up = 0, low = 0;
        bool bad = false;
    };
    std::vector<Part> part(static_cast<size_t>(nthr));
    auto run_rows = [&](auto&& check) -> RowErr {
        std::vector<RowErr> errs(static_cast<size_t>(nthr));
        host_parallel(nthr, [&](int t) {
            const int i0 = int((long long)n * t / nthr), i1 = int((long long)n * (t + 1) / nthr);
            for (int i = i0; i < i1; ++i)
                if (check(i, t, errs[size_t(t)]))
                    return;
        });
        RowErr best;
        for (auto& e : errs)
            if (e.code != ISING_OK && e.row < best.row)
                best = e;
        return best;
    };
    RowErr err = run_rows([&](int i, int t, RowErr& e) {
        long long b = std::llabs((long long)h[i]);
        long long eb = b;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            if (col[k] < 0 || col[k] >= n) {
                e = {i, ISING_ERR_INVALID_ARG, "column index out of range in row " + std::to_string(i)};
                return true;
            }
            if (col[k] == i) {
                e = {i, ISING_ERR_SELF_LOOP_OR_DUP, "self loop at spin " + std::to_string(i)};
                return true;
            }
            if (J[k] > 32767 || J[k] < -32767) {
                e = {i, ISING_ERR_INVALID_ARG, "|J| must be <= 32767"};
                return true;
            }
            ent[size_t(k)] = std::make_pair(col[k], J[k]);
            b += std::llabs((long long)J[k]);
            if (col[k] > i)
                eb += std::llabs((long long)J[k]);
        }
        std::sort(ent + row_ptr[i], ent + row_ptr[i + 1]);
        for (int k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k)
            if (ent[size_t(k)].first == ent[size_t(k) - 1].first) {
                e = {i, ISING_ERR_SELF_LOOP_OR_DUP, "repeated neighbour in row " + std::to_string(i)};
                return true;
            }
        Part& pt = part[size_t(t)];
        pt.km = std::max(pt.km, b);
        pt.eb += eb;
        return false;
    });
    if (err.code != ISING_OK)
        return fail(err.code, err.msg);
    // symmetry, fast test: every entry above the diagonal, (i, j, J) with
    // j > i, has its transpose (j, i, J), and there are as many entries below
    // the diagonal as above.  The transpose map is then one to one from the
    // upper entries onto the lower ones, so J is symmetric.
    auto has_transpose = [&](int i, int k) {
        const int j = ent[size_t(k)].first;
        const auto b = ent + row_ptr[j], en = ent + row_ptr[j + 1];
        const auto it = std::lower_bound(b, en, std::make_pair(i, INT32_MIN));
        return it != en && it->first == i && it->second == ent[size_t(k)].second;
    };
    host_parallel(nthr, [&](int t) {
        const int i0 = int((long long)n * t / nthr), i1 = int((long long)n * (t + 1) / nthr);
        long long up = 0, low = 0;
        bool bad = false;
        for (int i = i0; i < i1 && !bad; ++i)
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                if (ent[size_t(k)].first < i) {
                    ++low;
                    continue;
                }
                ++up;
                if (!has_transpose(i, k)) {
                    bad = true;
                    break;
                }
            }
        part[size_t(t)].up = up;
        part[size_t(t)].low = low;
        part[size_t(t)].bad = bad;
    });
    long long nup = 0, nlow = 0;
    bool any_bad = false;
    for (const Part& pt : part) {
        nup += pt.up;
        nlow += pt.low;
        any_bad |= pt.bad;
    }
    if (any_bad || nup != nlow) {
        // the error a row-by-row check of every entry meets first
        err = run_rows([&](int i, int, RowErr& e) {
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
                if (!has_transpose(i, k)) {
                    e = {i, ISING_ERR_ASYMMETRIC_J, "J(" + std::to_string(i) + "," +
                                                        std::to_string(ent[size_t(k)].first) +
                                                        ") has no equal transpose"};
                    return true;
                }
            return false;
        });
        return fail(err.code != ISING_OK ? err.code : ISING_ERR_ASYMMETRIC_J,
                    err.code != ISING_OK ? err.msg : std::string("J is not symmetric"));
    }
    long long km = 0, eb = 0;
    for (const Part& pt : part) {
        km = std::max(km, pt.km);
        eb += pt.eb;
    }
    if (kmax)
        *kmax = km;
    if (ebound)
        *ebound = eb;
    return ISING_OK;
}

// Checks that spin i = t*S + q has the spatial row of site q shifted to slice
// t plus the Trotter ring entries, with h and couplings identical in every
// slice.  Fills the slice tables.
int32_t extract_slices(ising_s* g)
{
    const int n = g->n, M = g->M, S = g->S;
    std::vector<std::vector<std::pair<int, int>>> sp(S);
    std::vector<int> jt(S, 0);
    // Spin i = t S + q: h equal to slice 0's, every coupling spatial (same
    // slice) or Trotter (same site, adjacent slice), the ring's Trotter
    // couplings present and equal, and (t > 0) the sorted spatial entries and
    // Trotter coupling equal to site q's in slice 0.  Slice 0 is checked
    // first, then the others against it, each phase in parallel chunks; of a
    // phase the error of the lowest spin is reported (the one a spin-by-spin
    // pass meets first).  Errors are raised on the calling thread.
    struct SpinErr {
        int i = INT32_MAX;
        std::string msg;
    };
    const int nthr = n >= 8192 ? host_threads() : 1;
    std::vector<SpinErr> errs(static_cast<size_t>(nthr));
    auto check = [&](int i, std::vector<std::pair<int, int>>& spat, SpinErr& e) -> bool {
        const int t = i / S, q = i - t * S;
        if (g->h[i] != g->h[q]) {
            e = {i, "declared slices differ in h at spin " + std::to_string(i)};
            return false;
        }
        spat.clear();
        int ntrot = 0, jtrot = 0;
        bool jt_ok = true;
        const int tm = (t + M - 1) % M, tp = (t + 1) % M;
        for (int k = g->row_ptr[i]; k < g->row_ptr[i + 1]; ++k) {
            const int c = g->col[k];
            const int tc = c / S, qc = c - tc * S;
            if (tc == t) {
                spat.emplace_back(qc, g->J[k]);
            } else if (qc == q && M >= 2 && (tc == tm || tc == tp)) {
                if (ntrot > 0 && g->J[k] != jtrot)
                    jt_ok = false;
                jtrot = g->J[k];
                ++ntrot;
            } else {
                e = {i, "spin " + std::to_string(i) + " has a coupling that is neither spatial nor Trotter"};
                return false;
            }
        }
        const int want = (M >= 3) ? 2 : (M == 2 ? 1 : 0);
        if (ntrot != want || !jt_ok) {
            e = {i, "spin " + std::to_string(i) + " lacks the Trotter ring couplings of the declared slices"};
            return false;
        }
        if (!std::is_sorted(spat.begin(), spat.end()))
            std::sort(spat.begin(), spat.end());
        if (t == 0) {
            sp[q] = spat;
            jt[q] = jtrot;
        } else if (spat != sp[q] || jtrot != jt[q]) {
            e = {i, "declared slices are not identical at spin " + std::to_string(i)};
            return false;
        }
        return true;
    };
    auto phase = [&](int lo, int hi) -> int32_t {
        for (auto& e : errs)
            e = SpinErr{};
        host_parallel(nthr, [&](int p) {
            std::vector<std::pair<int, int>> spat;
            const int i0 = lo + int((long long)(hi - lo) * p / nthr);
            const int i1 = lo + int((long long)(hi - lo) * (p + 1) / nthr);
            for (int i = i0; i < i1; ++i)
                if (!check(i, spat, errs[size_t(p)]))
                    return;
        });
        const SpinErr* best = nullptr;
        for (const auto& e : errs)
            if (e.i != INT32_MAX && (!best || e.i < best->i))
                best = &e;
        return best ? fail(ISING_ERR_INVALID_ARG, best->msg) : ISING_OK;
    };
    int32_t rc = phase(0, S);
    if (!rc && n > S)
        rc = phase(S, n);
    if (rc)
        return rc;
    (void)n;
    // slice wavefront levels: lev0(q) = 1 + max lev0(q') over spatial q' < q
    std::vector<int> lev(S, 0);
    int D0 = 0;
    for (int q = 0; q < S; ++q) {
        int l = 0;
        for (auto& e : sp[q])
            if (e.first < q)
                l = std::max(l, lev[e.first] + 1);
        lev[q] = l;
        D0 = std::max(D0, l + 1);
    }
    g->D0 = D0;
    g->D = D0 + M - 1;
    g->site.resize(S);
    for (int q = 0; q < S; ++q)
        g->site[q] = q;
    std::stable_sort(g->site.begin(), g->site.end(), [&](int a, int b) { return lev[a] < lev[b]; });
    g->pos.assign(S, 0);
    for (int p = 0; p < S; ++p)
        g->pos[g->site[p]] = p;
    g->lev0p.resize(S);
    g->jtau.resize(S);
    g->nbr_off.assign(S + 1, 0);
    g->nbr.clear();
    g->max_sp_deg = 0;
    g->max_sp_J = 0;
    for (int q = 0; q < S; ++q) {
        g->max_sp_deg = std::max(g->max_sp_deg, int(sp[q].size()));
        for (auto& e : sp[q])
            g->max_sp_J = std::max(g->max_sp_J, std::abs(e.second));
    }
    for (int p = 0; p < S; ++p) {
        const int q = g->site[p];
        g->lev0p[p] = lev[q];
        g->jtau[p] = jt[q];
        for (auto& e : sp[q])
            g->nbr.push_back((uint32_t(g->pos[e.first]) << 16) | (uint32_t(e.second) & 0xFFFFu));
        g->nbr_off[p + 1] = int(g->nbr.size());
    }
    // tracks: positions (in lev0 order) packed greedily into sequences whose
    // busy windows [lev0, lev0 + M) do not overlap; with equal window lengths
    // and sorted starts the earliest-freed track is the oldest one
    {
        std::vector<std::vector<int>> tr;
        std::vector<int> fifo;  // track indices in the order they free up
        size_t head = 0;
        std::vector<int> free_at;
        for (int p = 0; p < S; ++p) {
            const int start = g->lev0p[p];
            int k;
            if (head < fifo.size() && free_at[fifo[head]] <= start) {
                k = fifo[head++];
            } else {
                k = int(tr.size());
                tr.emplace_back();
                free_at.push_back(0);
            }
            tr[k].push_back(p);
            free_at[k] = start + M;
            fifo.push_back(k);
        }
        g->ntracks = int(tr.size());
        g->track_off_v.assign(1, 0);
        g->track_col.clear();
        for (auto& t : tr) {
            g->track_col.insert(g->track_col.end(), t.begin(), t.end());
            g->track_off_v.push_back(int(g->track_col.size()));
        }
    }
    // slots of the packed kernel: the same windows, each column (in lev0
    // order) into the lowest-numbered slot free at its start, so that the busy
    // slots of a level crowd the lowest numbers; a slot is free again at the
    // first level divisible by 4 at or after its column's window (the kernel
    // moves slots to their next column at those levels)
    {
        std::vector<std::vector<int>> sl;
        std::vector<int> free_at;
        for (int p = 0; p < S; ++p) {
            const int start = g->lev0p[p];
            size_t k = 0;
            while (k < free_at.size() && free_at[k] > start)
                ++k;
            if (k == free_at.size()) {
                sl.emplace_back();
                free_at.push_back(0);
            }
            sl[k].push_back(p);
            free_at[k] = (start + M + 3) & ~3;
        }
        g->nslots = int(sl.size());
        g->slot_off_v.assign(1, 0);
        g->slot_col_v.clear();
        for (auto& v : sl) {
            g->slot_col_v.insert(g->slot_col_v.end(), v.begin(), v.end());
            g->slot_off_v.push_back(int(g->slot_col_v.size()));
        }
        g->sp_bound = 0;
        for (int q = 0; q < S; ++q) {
            int b = std::abs(g->h[q]);
            for (auto& e : sp[q])
                b += std::abs(e.second);
            g->sp_bound = std::max(g->sp_bound, b);
        }
    }
    return ISING_OK;
}

// Word slots of the packed kernel's column words (a permutation of the
// positions; bank = slot mod 32).  A level's neighbour loads of a warp (one
// instruction per neighbour entry, one address per lane) take as many
// shared-memory wavefronts as the most-used bank has distinct words, so the
// slots are chosen by a greedy search over swaps that lowers the sum of those
// counts over one sweep's load instructions, simulated with the kernel's own
// slot schedule (a lane holds its slot's current column: the first one from
// the sweep's start, the next one from the last level divisible by 4 before
// its start; warps without a busy lane skip the level when a thread has one
// slot; long columns: the busy word of each column, all at one bank offset
// when S is a multiple of 32).  Deterministic; about 40 tries per column
// (a batch runs its instances' searches on the host threads).
std::vector<int> packed_word_slots(const ising_s* g, int T)
{
    const int S = g->S, M = g->M, D = g->D, ns = g->nslots;
    std::vector<int> slot(S);
    for (int p = 0; p < S; ++p)
        slot[p] = p;
    // long columns are stored word-major, so a word's bank is its slot's only
    // when S is a multiple of 32
    if (S < 64 || T <= 0 || (M > 32 && S % 32 != 0))
        return slot;
    const int rounds = (ns + T - 1) / T;
    const int NSP = rounds * T;
    // the load instructions of a sweep: distinct positions per (level, warp,
    // round, entry); -1 stands for word 0 (padding, idle rounds)
    std::vector<int> cur(NSP, -1), idx(NSP, 0);
    for (int sl = 0; sl < ns; ++sl)
        if (g->slot_off_v[sl] < g->slot_off_v[sl + 1])
            cur[sl] = g->slot_col_v[g->slot_off_v[sl]];
    std::vector<int> ioff(1, 0), iword;  // instruction i: iword[ioff[i] .. ioff[i + 1])
    std::vector<char> iw0;               // instruction reads word 0
    std::vector<int> tmp;
    for (int l = 0; l < D; ++l) {
        if ((l & 3) == 0)
            for (int sl = 0; sl < ns; ++sl) {
                const int k = g->slot_off_v[sl] + idx[sl] + 1;
                if (k < g->slot_off_v[sl + 1] && (g->lev0p[g->slot_col_v[k]] & ~3) <= l) {
                    ++idx[sl];
                    cur[sl] = g->slot_col_v[k];
                }
            }
        for (int c = 0; c < rounds; ++c)
            for (int w0 = 0; w0 < T; w0 += 32) {
                bool busy = rounds > 1;
                for (int i = 0; i < 32 && !busy; ++i) {
                    const int p = cur[c * T + w0 + i];
                    busy = p >= 0 && unsigned(l - g->lev0p[p]) < unsigned(M);
                }
                if (!busy)
                    continue;
                for (int e = 0; e < isg::packed_detail::kMaxDeg; ++e) {
                    tmp.clear();
                    char w0flag = 0;
                    for (int i = 0; i < 32; ++i) {
                        const int p = cur[c * T + w0 + i];
                        if (p < 0 || e >= g->nbr_off[p + 1] - g->nbr_off[p]) {
                            w0flag = 1;
                            continue;
                        }
                        tmp.push_back(int(g->nbr[g->nbr_off[p] + e] >> 16));
                    }
                    std::sort(tmp.begin(), tmp.end());
                    tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
                    iword.insert(iword.end(), tmp.begin(), tmp.end());
                    ioff.push_back(int(iword.size()));
                    iw0.push_back(w0flag);
                }
            }
    }
    const int ni = int(iw0.size());
    if (ni == 0)
        return slot;
    // per instruction: words per bank, how many banks hold each count, max
    std::vector<std::vector<int>> occ(S);
    std::vector<int16_t> cnt(size_t(ni) * 32, 0), hist(size_t(ni) * 33, 0), mx(ni, 0);
    for (int i = 0; i < ni; ++i) {
        int16_t* ci = cnt.data() + size_t(i) * 32;
        if (iw0[i])
            ci[0] += 1;
        for (int k = ioff[i]; k < ioff[i + 1]; ++k) {
            occ[iword[k]].push_back(i);
            ci[iword[k] & 31] += 1;
        }
        for (int b = 0; b < 32; ++b)
            hist[size_t(i) * 33 + ci[b]] += 1;
        mx[i] = *std::max_element(ci, ci + 32);
    }
    auto move = [&](int i, int from, int to) {  // one word of instruction i from bank `from` to `to`
        int16_t* ci = cnt.data() + size_t(i) * 32;
        int16_t* hi = hist.data() + size_t(i) * 33;
        hi[ci[from]] -= 1;
        ci[from] -= 1;
        hi[ci[from]] += 1;
        if (hi[mx[i]] == 0)
            mx[i] -= 1;
        hi[ci[to]] -= 1;
        ci[to] += 1;
        hi[ci[to]] += 1;
        if (ci[to] > mx[i])
            mx[i] = ci[to];
    };
    uint64_t st = 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        st ^= st << 13;
        st ^= st >> 7;
        st ^= st << 17;
        return st;
    };
    std::vector<int> stamp(ni, -1), aff;
    std::vector<int16_t> old_mx(ni, 0);
    const int iters = 40 * S;
    for (int it = 0; it < iters; ++it) {
        const int a = int(next() % uint64_t(S)), b = int(next() % uint64_t(S));
        const int A = slot[a] & 31, B = slot[b] & 31;
        if (A == B)
            continue;
        aff.clear();
        for (const std::vector<int>* o : {&occ[a], &occ[b]})
            for (int i : *o)
                if (stamp[i] != it) {
                    stamp[i] = it;
                    old_mx[i] = mx[i];
                    aff.push_back(i);
                }
        for (int i : occ[a])
            move(i, A, B);
        for (int i : occ[b])
            move(i, B, A);
        int d = 0;
        for (int i : aff)
            d += mx[i] - old_mx[i];
        if (d <= 0) {
            std::swap(slot[a], slot[b]);
        } else {
            for (int i : occ[b])
                move(i, A, B);
            for (int i : occ[a])
                move(i, B, A);
        }
    }
    return slot;
}

// The search's result per model and block shape (the last few, compared in
// full): handles of the same model made one after another skip the search.
std::vector<int> packed_word_slots_cached(const ising_s* g, int T)
{
    std::vector<int> key = {g->S, g->M, g->D, g->nslots, T};
    key.insert(key.end(), g->lev0p.begin(), g->lev0p.end());
    key.insert(key.end(), g->nbr_off.begin(), g->nbr_off.end());
    for (uint32_t e : g->nbr)
        key.push_back(int(e >> 16));
    key.insert(key.end(), g->slot_off_v.begin(), g->slot_off_v.end());
    key.insert(key.end(), g->slot_col_v.begin(), g->slot_col_v.end());
    static std::mutex mu;
    static std::vector<std::pair<std::vector<int>, std::vector<int>>> cache;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto& e : cache)
            if (e.first == key)
                return e.second;
    }
    std::vector<int> ws = packed_word_slots(g, T);
    std::lock_guard<std::mutex> lk(mu);
    if (cache.size() >= 4)
        cache.erase(cache.begin());
    cache.emplace_back(std::move(key), ws);
    return ws;
}

// The packed kernel's table buffer: column descriptors [S][16] (lev0 | site
// << 16, byte offset of the column's own word (4 x its word slot), 2 Jtau, the field constant
// h_q - sum_j J_qj - 2 Jtau, six byte offsets of the spatial neighbours'
// words, their six 2 J; missing neighbours padded with word 0 and J = 0),
// positions [S], slot offsets [nslots + 1], slot columns [S], each
// part padded to 16 bytes.
std::vector<uint32_t> packed_tables(const ising_s* g, int T)
{
    using isg::packed_detail::kDescWords;
    using isg::packed_detail::kMaxDeg;
    const int S = g->S;
    const std::vector<int> ws = packed_word_slots_cached(g, T);
    auto pad4 = [](size_t n) { return (n + 3) & ~size_t(3); };
    std::vector<uint32_t> pk(isg::packed_detail::packed_table_bytes(S, g->nslots) / 4, 0u);
    for (int p = 0; p < S; ++p) {
        uint32_t* d = pk.data() + size_t(p) * kDescWords;
        const int jt2 = 2 * g->jtau[p];
        long long c = g->h[g->site[p]] - jt2;
        d[0] = uint32_t(g->lev0p[p]) | (uint32_t(g->site[p]) << 16);
        d[1] = 4u * uint32_t(ws[p]);  // long columns: their first word (word w is S words further on per w)
        d[2] = uint32_t(jt2);
        const int e0 = g->nbr_off[p], deg = g->nbr_off[p + 1] - e0;
        for (int e = 0; e < kMaxDeg; ++e) {
            if (e >= deg) {  // word 0 with J = 0: one word for all such loads of a warp
                d[4 + e] = 0u;
                d[10 + e] = 0u;
                continue;
            }
            const uint32_t en = g->nbr[e0 + e];
            const int pj = int(en >> 16), J = int(int16_t(en & 0xFFFFu));
            c -= J;
            d[4 + e] = 4u * uint32_t(ws[pj]);
            d[10 + e] = uint32_t(2 * J);
        }
        d[3] = uint32_t(int32_t(c));
    }
    size_t o = size_t(S) * kDescWords;
    for (int q = 0; q < S; ++q)
        pk[o + q] = uint32_t(g->pos[q]);
    o += pad4(S);
    for (int k = 0; k <= g->nslots; ++k)
        pk[o + k] = uint32_t(g->slot_off_v[k]);
    o += pad4(size_t(g->nslots) + 1);
    for (int i = 0; i < S; ++i)
        pk[o + i] = uint32_t(g->slot_col_v[i]);
    return pk;
}

// --------------------------------------------------- launch configuration
SweepArgs base_args(ising_s* g);

// The register-resident kernel keeps up to 8 columns per thread; it needs
// M <= 32, the slice tables in shared memory and spatial degree <= 255.
// The packed kernel generates its sweep words itself (two extra warps per
// block, two-sweep word buffer: MT19937 streams or Philox blocks); the
// separate generator then only makes MT19937's swap-stream words.
bool packed_gen(const ising_s* g) { return g->use_packed; }

int kernel_variant(const ising_s* g)
{
    if (g->use_packed)
        return 5;
    return g->use_track ? 2 : (g->use_lean ? (g->lean_long ? 4 : (g->lean_small ? 3 : 1)) : 0);
}

// The packed kernel's model limits: M in {8, 16, 32} (the column in one
// register, whole 4-word blocks) or a multiple of 32 up to 1024 (long columns:
// M / 32 words, the busy one in a register), spatial degree <= 6,
// |J| <= 127, positions and levels in 16 bits, plain couplings, one replica
// per block and no opt-out.
bool packed_eligible(const ising_s* g)
{
    const bool long_cols = g->M > 32 && g->M % 32 == 0 && g->M <= 1024 && g->S * (g->M / 32) < (1 << 20);
    return (g->M == 8 || g->M == 16 || g->M == 32 || long_cols) && g->max_sp_deg <= 6 && g->max_sp_J <= 127 &&
           g->S < 65536 && g->D < 65536 && g->nslots >= 1 && !g->split &&
           g->G_req <= 1 && !g->packed_off && !g->lean_off && !g->fast_off && !g->track_on &&
           (g->T_req == 0 || g->T_req == 32 || g->T_req == 64 || g->T_req == 128 || g->T_req == 256);
}

// Configure the packed kernel: sweep threads per block (one to eight warps;
// automatic: the fewest whole warps that give every slot its own thread, or
// four warps of several rounds beyond 256 slots), slot rounds per thread,
// two generator warps with MT19937, shared memory and the persistent check.
bool choose_packed(ising_s* g)
{
    if (!packed_eligible(g))
        return false;
    const int T = g->T_req > 0 ? g->T_req : (g->nslots <= 256 ? ((g->nslots + 31) / 32) * 32 : 128);
    const int rounds = (g->nslots + T - 1) / T;
    if (T > 128 && rounds > 1)
        return false;  // the instantiations with more than one round allow 128 threads
    int rmax = 0;
    for (int r : isg::kPackedRounds)
        if (rounds <= r) {
            rmax = r;
            break;
        }
    if (rmax == 0)
        return false;
    if (g->M > 32) {  // long columns: instantiations of one and two rounds
        if (rmax > 2)
            return false;
        rmax += isg::kPackedLong;
    }
    if (!g->d_pk) {
        const std::vector<uint32_t> pk = packed_tables(g, T);
        if (upload(&g->d_pk, pk) != ISING_OK)
            return false;
        g->pk_bytes = uint32_t(pk.size() * 4);
    }
    SweepArgs a = base_args(g);
    a.G = 1;
    a.gen = kPackedGenWarps;
    // MT19937: stage 4 slices per generator store, or 2 where the blocks of
    // a ladder would otherwise not all be resident (16 S bytes -> 8 S)
    int gsl = 4;
    a.gen_slices = 4;
    const int sw0 = a.swap_every;
    size_t plain = packed_smem_bytes(a, T);
    a.swap_every = 1;
    size_t fused = packed_smem_bytes(a, T);
    const size_t lim = sweep_max_dynamic_smem() ? sweep_max_dynamic_smem() : 200 * 1024;
    if (g->rng == ISING_RNG_MT19937) {
        int per4 = 0;
        const bool ok4 = fused <= lim && fast_max_blocks_per_sm(g->field_bits, rmax, g->rng, T + 32 * a.gen, fused,
                                                               &per4, 5) == cudaSuccess;
        if (!(ok4 && (long long)per4 * g_num_sms >= g->R)) {
            gsl = 2;
            a.gen_slices = 2;
            a.swap_every = sw0;
            plain = packed_smem_bytes(a, T);
            a.swap_every = 1;
            fused = packed_smem_bytes(a, T);
        }
    }
    if (plain > lim)
        return false;
    // A ladder that cannot be resident at once is throughput-bound rather than
    // bound by one replica's chain of levels; there the lean kernel's
    // small-block build is faster (65536 replicas of 4096 spins: 1.18e11
    // against 1.05e11 attempts/s), so the packed kernel is chosen
    // automatically only for resident ladders.  The handle is changed only
    // when the packed kernel is taken.
    int per_sm = 0;
    const bool occ = fused <= lim && fast_max_blocks_per_sm(g->field_bits, rmax, g->rng, T + 32 * a.gen, fused,
                                                           &per_sm, 5) == cudaSuccess;
    const bool resident = occ && (long long)per_sm * g_num_sms >= g->R;
    if (!resident && g->T_req == 0)
        return false;
    g->use_packed = true;
    g->use_fast = true;
    g->gen_slices = gsl;
    g->G = 1;
    g->T = T;
    g->blocks = g->R;
    g->fast_cmax = rmax;
    g->fast_smem = plain;
    g->smem_fused = fused;
    g->smem = plain;
    g->persistent_ok = resident && g_coop && g->allow_persistent && g->R <= 16384;
    return true;
}

// slice counts of the lean kernel: a power of two from 4 to 32 (the column in
// one register), or a multiple of 32 up to 1024 (long columns, M / 32 words)
bool lean_slices(int M) { return M == 4 || M == 8 || M == 16 || M == 32 || (M % 32 == 0 && M <= 1024); }

// The lean kernel's model limits (one replica per block; the block size is
// checked when the launch is chosen).
bool lean_eligible(const ising_s* g)
{
    return lean_slices(g->M) && g->max_sp_deg <= 6 && g->max_sp_J <= 63 &&
           g->G_req <= 1 && !g->lean_off && !g->fast_off;
}

// The track kernel (opt-in, ISING_LAUNCH_TRACK) and its limits (lean's, with
// one thread per track): power-of-two M in 4..32, spatial degree <= 6,
// |J| <= 63, at most 512 tracks, and the block size left to the library.
bool track_eligible(const ising_s* g)
{
    return (g->M == 4 || g->M == 8 || g->M == 16 || g->M == 32) && g->max_sp_deg <= 6 &&
           g->max_sp_J <= 63 && g->ntracks >= 1 && ((g->ntracks + 31) / 32) * 32 <= 512 && g->T_req <= 0 &&
           g->track_on && !g->lean_off && !g->fast_off;
}

void choose_fast(ising_s* g)
{
    g->use_fast = false;
    g->use_packed = false;
    g->use_lean = false;
    g->lean_small = false;
    g->lean_long = false;
    g->use_track = false;
    g->persistent_ok = false;
    if (choose_packed(g))
        return;
    // M > 32: only the lean kernel's long-column instantiation (M a multiple of 32)
    const bool long_cols = g->M > 32;
    if ((long_cols && !lean_slices(g->M)) || !g->tables_smem || g->max_sp_deg > 255 || g->fast_off)
        return;
    const long long C = ((long long)g->S * g->G + g->T - 1) / g->T;
    int cmax = 0;
    for (int m : {1, 2, 4, 8})
        if (C <= m) {
            cmax = m;
            break;
        }
    if (cmax == 0 || g->T > (cmax <= 2 ? 1024 : (cmax == 4 ? 512 : 256)))
        return;
    // lean variant: one replica per block, power-of-two M >= 4, small degree
    // and couplings, at most 4 columns per thread within its register budget
    g->use_lean = g->G == 1 && lean_slices(g->M) && g->max_sp_deg <= 6 && g->max_sp_J <= 63 &&
                  cmax <= (long_cols ? 2 : 4) &&
                  g->T <= (cmax <= 1 ? 1024 : (cmax == 2 ? 512 : 256)) && !g->lean_off &&
                  (g->rng == ISING_RNG_MT19937 || (g->ntracks >= 1 && g->ntracks <= g->T));
    if (long_cols && !g->use_lean)
        return;  // the register-resident fast kernel holds a column in one word
    if (g->split && !g->use_lean)
        return;  // split couplings: the lean kernel only
    g->lean_long = long_cols;
    // track variant: the lean kernel's limits with the columns walked as
    // tracks, one thread per track (when the block size is left automatic)
    const int T_track = ((g->ntracks + 31) / 32) * 32;
    if (g->G == 1 && !long_cols && !g->split && track_eligible(g)) {
        SweepArgs t = base_args(g);
        t.G = 1;
        const size_t sm = fast_smem_bytes(t, g->field_bits, 2, T_track);
        if (sm != size_t(-1)) {  // the fused (PT) layout is checked below with persistence
            g->use_track = true;
            g->use_lean = false;
            g->T = T_track;
            cmax = 1;
        }
    }
    // two columns per thread in blocks of at most 128 threads: the small-block
    // lean instantiation (eight resident blocks per SM)
    g->lean_small = g->use_lean && !long_cols && cmax == 2 && g->T <= kLeanSmallThreads;
    const int variant = kernel_variant(g);
    SweepArgs a = base_args(g);
    const size_t smem = fast_smem_bytes(a, g->field_bits, variant, g->T);
    if (smem == size_t(-1))
        return;
    g->use_fast = true;
    g->fast_cmax = cmax;
    g->fast_smem = smem;
    a.swap_every = 1;
    g->smem_fused = fast_smem_bytes(a, g->field_bits, variant, g->T);
    if (!g_coop || !g->allow_persistent || g->smem_fused == size_t(-1) || g->R > 16384)
        return;
    int per_sm = 0;
    if (fast_max_blocks_per_sm(g->field_bits, cmax, g->rng, g->T, g->smem_fused, &per_sm, variant,
                               g->split) != cudaSuccess)
        return;
    g->persistent_ok = (long long)per_sm * g_num_sms >= g->blocks;
}

SweepArgs base_args(ising_s* g)
{
    SweepArgs a{};
    a.S = g->S;
    a.M = g->M;
    a.W = g->W;
    a.N = g->n;
    a.D0 = g->D0;
    a.D = g->D;
    a.Mp = g->Mp;
    a.K = g->K;
    a.G = g->G;
    a.R = g->R;
    a.tables_smem = g->tables_smem;
    a.thr_smem = g->thr_smem;
    a.nbr_count = int(g->nbr.size());
    a.nbr_off = g->d_nbr_off;
    a.nbr = g->d_nbr;
    a.jtau = g->d_jtau;
    a.lev0 = g->d_lev0;
    a.site = g->d_site;
    a.pos = g->d_pos;
    a.spins = g->d_spins;
    a.fields = g->d_fields;
    a.E = g->d_E;
    a.temp_of_slot = g->d_temp;
    a.thr = g->d_thr;
    a.rng = g->rng;
    a.seed = g->seed;
    a.inst = g->inst;
    a.counters = g->d_counters;
    a.done_blocks = g->d_done;
    a.err = g->d_err;
    a.wbuf_sweep_stride = (long long)g->R * g->S * g->Mp;
    int lg = 0;
    while ((1 << lg) < g->G)
        ++lg;
    a.lg_G = lg;
    a.swap_every = 0;
    a.slot_of_temp = g->d_slot;
    a.temp_of_slot_out = g->d_temp;
    a.swap_acc = g->d_swap_acc;
    a.swthr = g->d_swthr;
    a.swoff = g->d_swoff;
    a.swlen = g->d_swlen;
    a.swbuf = g->d_swbuf;
    a.maxpairs = g->maxpairs;
    a.E_pub = g->d_Epub;
    a.gridbar = g->d_gridbar;
    a.track_off = g->d_track_off;
    a.track_col = g->d_track_col;
    a.ntracks = g->ntracks;
    a.stage_words = g->stage_words;
    // busy columns of a level form a contiguous range of positions no longer
    // than ntracks (the widest level); a thread's columns are T positions apart
    a.one_active = (g->ntracks >= 1 && g->ntracks <= g->T) ? 1 : 0;
    a.split = g->split ? 1 : 0;
    a.split_ks = g->split_ks;
    a.C = g->d_C;
    a.C_pub = g->d_Cpub;
    a.dbeta = g->d_dbeta;
    a.dK = g->d_dK;
    a.pk = g->d_pk;
    a.pk_bytes = g->pk_bytes;
    a.nslots = g->nslots;
    a.field_bits = g->field_bits;
    a.gen = packed_gen(g) ? kPackedGenWarps : 0;
    a.gen_slices = g->gen_slices;
    a.mtring = g->d_mtring;
    a.mtpos = g->d_mtpos;
    a.sweep_threads = g->T;
    return a;
}

int32_t choose_launch(ising_s* g)
{
    if (packed_eligible(g) && choose_packed(g)) {
        // the packed kernel sizes its own blocks (one replica per block)
        g->use_lean = g->lean_small = g->lean_long = g->use_track = false;
        g->tables_smem = 1;
        g->thr_smem = 1;
        g->stage_words = 0;
        g->cmax = 1;
        return ISING_OK;
    }
    const int sms = g_num_sms > 0 ? g_num_sms : 148;
    const size_t kMaxSmem = sweep_max_dynamic_smem() ? sweep_max_dynamic_smem() : 200 * 1024;
    const long long table_bytes = 4LL * (4 * g->S + 1) + 4LL * (long long)g->nbr.size();
    std::vector<int> Gs;
    if (g->G_req > 0) {
        Gs.push_back(g->G_req);
    } else if (track_eligible(g) || lean_eligible(g)) {
        Gs.push_back(1);  // the track and lean kernels run one replica per block
    } else {
        for (int G : {8, 4, 2, 1})
            if ((long long)((g->R + G - 1) / G) >= 2LL * sms || G == 1)
                Gs.push_back(G);
    }
    for (int G : Gs) {
        for (int tables_smem : {1, 0}) {
            if (tables_smem && table_bytes > 96 * 1024)
                continue;
            SweepArgs a = base_args(g);
            a.G = G;
            a.tables_smem = tables_smem;
            a.thr_smem = (4LL * G * g->K <= 16 * 1024) ? 1 : 0;
            // MT19937 words are staged (measured 1.4x on the 96 x 256-layer model);
            // Philox words are computed per visit, in parallel across the level
            a.stage_words = g->rng == ISING_RNG_MT19937 ? 1 : 0;
            size_t smem = sweep_smem_bytes(a, g->field_bits);
            if (smem > kMaxSmem) {
                a.stage_words = 0;
                smem = sweep_smem_bytes(a, g->field_bits);
            }
            if (smem > kMaxSmem)
                continue;
            int T = g->T_req;
            if (T <= 0) {
                // four columns per thread for the register-resident kernels (M <= 32);
                // one per thread for the generic kernel, whose per-level loop over a
                // thread's columns is serial (the paper-shaped 96 x 256 model: 2.2x)
                long long want = g->M > 32 ? (long long)g->S * G : ((long long)g->S * G + 3) / 4;
                if (G == 1 && g->M <= 32) {
                    // a ladder too large to stay resident (no fused PT) runs two
                    // columns per thread (cfg3, 65536 replicas: 1.3x over four);
                    // at least as many threads as the widest level has busy columns
                    // (the lean kernel's Philox state is per thread)
                    if ((long long)g->R > 4LL * sms)
                        want = ((long long)g->S + 1) / 2;
                    want = std::max<long long>(want, g->ntracks);
                }
                T = int(std::min<long long>(1024, std::max<long long>(32, ((want + 31) / 32) * 32)));
            }
            if (T % 32 != 0 || T > 1024 || T % G != 0)
                return fail(ISING_ERR_INVALID_ARG, "threads per block must be a multiple of 32 and of G, <= 1024");
            const long long C = ((long long)g->S * G + T - 1) / T;
            const int cmax = sweep_cmax_for(int(std::min<long long>(C, 64)));
            if (cmax == 0) {
                if (g->T_req > 0)
                    return fail(ISING_ERR_UNSUPPORTED, "more than 32 columns per thread");
                continue;
            }
            g->G = G;
            g->T = T;
            g->cmax = cmax;
            g->tables_smem = tables_smem;
            g->thr_smem = a.thr_smem;
            g->stage_words = a.stage_words;
            g->smem = smem;
            g->blocks = (g->R + G - 1) / G;
            choose_fast(g);
            return ISING_OK;
        }
    }
    return fail(ISING_ERR_UNSUPPORTED, "replica state of one block does not fit in shared memory");
}

// ------------------------------------------------------- launch planning
struct Op {
    enum Kind { GEN, SWEEP, PT, FUSED } kind;
    int sweeps;   // GEN: sweeps of words; SWEEP/FUSED: sweeps
    int passes;   // GEN: passes of swap words; FUSED: sweeps between PT passes
    int offset;   // SWEEP: sweep offset into wbuf; PT: pass offset into swbuf
};

std::vector<Op> plan(ising_s* g, long long n, int swap_every, long long cap)
{
    std::vector<Op> ops;
    const bool mt = g->rng == ISING_RNG_MT19937;
    const bool own = packed_gen(g);  // sweep words generated by the sweep kernel
    long long done = 0;
    if (n <= 0 && swap_every == -1) {
        // a lone PT pass
        if (mt)
            ops.push_back({Op::GEN, 0, 1, 0});
        ops.push_back({Op::PT, 0, 0, 0});
        return ops;
    }
    if (g->persistent_ok && swap_every > 0 && swap_every <= cap) {
        // whole groups of `swap_every` sweeps run in persistent launches with
        // the PT pass fused; a trailing partial group has no PT pass
        const long long per = (cap / swap_every) * swap_every;
        while (n - done >= swap_every) {
            const long long m = std::min(per, ((n - done) / swap_every) * swap_every);
            if (mt)
                ops.push_back({Op::GEN, own ? 0 : int(m), int(m / swap_every), 0});
            ops.push_back({Op::FUSED, int(m), swap_every, 0});
            done += m;
        }
        if (done < n) {
            if (mt && !own)
                ops.push_back({Op::GEN, int(n - done), 0, 0});
            ops.push_back({Op::SWEEP, int(n - done), 0, 0});
        }
        return ops;
    }
    while (done < n) {
        std::vector<Op> chunk;
        long long cs = 0;
        int cp = 0;
        while (done < n && cs < cap) {
            const long long to_pt = swap_every > 0 ? swap_every - (done % swap_every) : n - done;
            const long long m = std::min({to_pt, n - done, cap - cs});
            chunk.push_back({Op::SWEEP, int(m), 0, int(cs)});
            cs += m;
            done += m;
            if (swap_every > 0 && done % swap_every == 0) {
                chunk.push_back({Op::PT, 0, 0, cp});
                ++cp;
            }
        }
        if (mt && (!own || cp > 0))
            ops.push_back({Op::GEN, own ? 0 : int(cs), cp, 0});
        ops.insert(ops.end(), chunk.begin(), chunk.end());
    }
    return ops;
}

long long words_cap(ising_s* g, long long n)
{
    if (g->rng != ISING_RNG_MT19937)
        return std::max<long long>(n, 1);
    if (packed_gen(g))  // only the swap stream's words are made ahead: up to 256 MB of them
        return std::max<long long>(
            1, std::min<long long>(std::max<long long>(n, 1), (256LL << 20) / (4LL * std::max(g->maxpairs, 1))));
    const long long per_sweep = (long long)g->R * g->S * g->Mp * 4;
    return std::max<long long>(1, std::min<long long>(std::max<long long>(n, 1), g->word_budget / per_sweep));
}

int32_t ensure_buffers(ising_s* g, long long cap_sweeps, long long cap_passes)
{
    if (packed_gen(g))
        cap_sweeps = 2;  // the sweep kernel's two-sweep word buffer (both generators)
    else if (g->rng != ISING_RNG_MT19937)
        return ISING_OK;
    if (cap_sweeps > g->wbuf_cap) {
        big_free(g->d_wbuf);
        // fully written by the generator before any sweep reads it: no zero fill
        int32_t rc = big_alloc(&g->d_wbuf, size_t(cap_sweeps) * g->R * g->S * g->Mp);
        if (rc)
            return rc;
        g->wbuf_cap = cap_sweeps;
    }
    if (g->rng == ISING_RNG_MT19937 && cap_passes > g->swbuf_cap) {
        dfree(g->d_swbuf);
        int32_t rc = dalloc(&g->d_swbuf, size_t(cap_passes) * std::max(g->maxpairs, 1));
        if (rc)
            return rc;
        g->swbuf_cap = cap_passes;
    }
    return ISING_OK;
}

// Kernel argument records of one planned op (also used by batched launches).
MtGenArgs gen_args(ising_s* g, const Op& op, int* blocks)
{
    MtGenArgs a{};
    a.ring = g->d_mtring;
    a.pos = g->d_mtpos;
    a.R = g->R;
    a.mode = 0;
    a.nwords = (long long)op.sweeps * g->n;
    a.N = g->n;
    a.S = g->S;
    a.M = g->M;
    a.Mp = g->Mp;
    a.pos_of_site = g->d_pos;
    a.wbuf = g->d_wbuf;
    a.wbuf_sweep_stride = (long long)g->R * g->S * g->Mp;
    a.do_swap = op.passes > 0;
    a.swap_passes = op.passes;
    a.swbuf = g->d_swbuf;
    a.maxpairs = g->maxpairs;
    a.counters = g->d_counters;
    // blocks: the R replica streams (when sweep words are needed), then the
    // swap stream (index R) when passes are needed
    a.first_stream = op.sweeps > 0 ? 0 : g->R;
    *blocks = (op.sweeps > 0 ? g->R : 0) + (a.do_swap ? 1 : 0);
    return a;
}

SweepArgs sweep_args(ising_s* g, const Op& op)
{
    SweepArgs a = base_args(g);
    a.nsweeps = op.sweeps;
    a.inst_blocks = g->blocks;
    if (op.kind == Op::FUSED) {
        a.swap_every = op.passes;
        a.wbuf = g->d_wbuf;
    } else {
        a.wbuf = (g->d_wbuf && !a.gen) ? g->d_wbuf + size_t(op.offset) * a.wbuf_sweep_stride : g->d_wbuf;
    }
    return a;
}

PtArgs pt_args(ising_s* g, const Op& op)
{
    PtArgs a{};
    a.R = g->R;
    a.E = g->d_E;
    a.temp_of_slot = g->d_temp;
    a.slot_of_temp = g->d_slot;
    a.swap_acc = g->d_swap_acc;
    a.counters = g->d_counters;
    a.swthr = g->d_swthr;
    a.swoff = g->d_swoff;
    a.swlen = g->d_swlen;
    a.rng = g->rng;
    a.seed = g->seed;
    a.inst = g->inst;
    a.swbuf = g->d_swbuf;
    a.maxpairs = g->maxpairs;
    a.pass_rel = op.offset;
    a.split = g->split ? 1 : 0;
    a.C = g->d_C;
    a.dbeta = g->d_dbeta;
    a.dK = g->d_dK;
    return a;
}

int32_t enqueue(ising_s* g, const std::vector<Op>& ops, cudaStream_t st)
{
    for (const Op& op : ops) {
        cudaError_t e = cudaSuccess;
        const bool is_sweep = op.kind == Op::SWEEP || op.kind == Op::FUSED;
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (is_sweep && g->profiling) {
            CK(cudaEventCreate(&ev0));
            CK(cudaEventCreate(&ev1));
            CK(cudaEventRecord(ev0, st));
        }
        if (op.kind == Op::GEN) {
            int blocks = 0;
            const MtGenArgs a = gen_args(g, op, &blocks);
            if (blocks > 0)
                e = launch_mt_gen(a, blocks, st);
        } else if (op.kind == Op::SWEEP) {
            const SweepArgs a = sweep_args(g, op);
            if (g->use_fast)
                e = launch_fast(a, g->field_bits, g->fast_cmax, g->T, g->blocks, g->fast_smem, false, st,
                                kernel_variant(g));
            else
                e = launch_sweep(a, g->field_bits, g->cmax, g->T, g->blocks, g->smem, st);
        } else if (op.kind == Op::FUSED) {
            const SweepArgs a = sweep_args(g, op);
            e = cudaMemsetAsync(g->d_gridbar, 0, sizeof(unsigned), st);
            if (e == cudaSuccess)
                e = launch_fast(a, g->field_bits, g->fast_cmax, g->T, g->blocks, g->smem_fused, true, st,
                                kernel_variant(g));
        } else {
            e = launch_pt(pt_args(g, op), st);
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "kernel launch");
        if (ev1) {
            CK(cudaEventRecord(ev1, st));
            g->ev_pending.emplace_back(ev0, ev1);
        }
    }
    return ISING_OK;
}

// kernels launched by a plan (GEN with nothing to do launches nothing)
std::pair<long long, long long> count_kernels(ising_s* g, const std::vector<Op>& ops)
{
    long long all = 0, sweeps = 0;
    for (const Op& op : ops) {
        if (op.kind == Op::GEN)
            all += (op.sweeps > 0 || op.passes > 0) ? 1 : 0;
        else if (op.kind == Op::PT)
            all += 1;
        else {
            all += 1;
            sweeps += 1;
        }
    }
    (void)g;
    return {all, sweeps};
}

int32_t check_device_error(ising_s* g)
{
    int err = 0;
    CK(cudaMemcpyAsync(&err, g->d_err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (err == kErrTimeout)
        return fail(ISING_ERR_TIMEOUT, "a bounded device wait gave up");
    if (err != 0)
        return fail(ISING_ERR_CUDA, "device error flag " + std::to_string(err));
    return ISING_OK;
}

}  // namespace

// Launch description of a handle's sweep kernels, for entry points defined in
// other translation units (noalloc.cu).  Returns NOT_INITIALISED /
// UNSUPPORTED when the handle has no register-resident fused path.
int32_t isg_fused_launch(ising_t g, isg::FusedLaunch* out)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (!g->use_fast || !g->persistent_ok)
        return fail(ISING_ERR_UNSUPPORTED,
                    "this model/ladder has no persistent fused launch (replicas do not all fit on the GPU)");
    if (g->split)
        return fail(ISING_ERR_UNSUPPORTED, "split couplings run through ising_run / ising_sweep only");
    out->args = base_args(g);
    out->field_bits = g->field_bits;
    out->cmax = g->fast_cmax;
    out->threads = g->T;
    out->blocks = g->blocks;
    out->smem_plain = g->fast_smem;
    out->smem_fused = g->smem_fused;
    out->variant = kernel_variant(g);
    out->stream = g->stream;
    out->R = g->R;
    out->rng = g->rng;
    return ISING_OK;
}

int32_t isg_fail(int32_t code, const char* msg) { return fail(code, msg); }

int isg_num_sms() { return g_num_sms > 0 ? g_num_sms : 1; }

bool isg_alloc_allowed(size_t bytes) { return alloc_allowed(bytes); }

bool isg_pt_ok(const ising_s* g) { return g->pt_ok; }

void isg_count_launches(ising_t g, long long all, long long sweeps)
{
    g->n_launches += all;
    g->n_sweep_launches += sweeps;
}

int32_t isg_device_setup()
{
    const cudaError_t e = device_setup();
    return e == cudaSuccess ? ISING_OK : cuda_fail(e, "device setup");
}

// ====================================================================== ABI
namespace {

// Swap thresholds S_k(d) = floor(2^32 exp(-(b_{k+1}-b_k) d)) for 1 <= d < len_k
// of every pair k of a ladder, flattened (pair k's table starts at off[k]).
struct SwapTables {
    std::vector<uint32_t> thr;
    std::vector<long long> off;
    std::vector<int> len;
    bool pt_ok = true;  // false when the tables would exceed 2^28 entries
};

std::shared_ptr<const SwapTables> build_swap_tables(const double* betas, int R, long long dmax)
{
    auto out = std::make_shared<SwapTables>();
    std::vector<long long>& swoff = out->off;
    std::vector<int>& swlen = out->len;
    std::vector<uint32_t>& swthr = out->thr;
    swoff.assign(std::max(R - 1, 1), 0);
    swlen.assign(std::max(R - 1, 1), 1);
    // S_k(d) is zero once 2^32 exp(-db d) < 1, i.e. beyond d = 32 ln 2 / db
    // (+1 for the rounding of the FP64 expression).  When these bounds keep
    // the tables within 2^28 entries, each pair's table is written in
    // parallel at an offset given by the bounds, with the same expression and
    // stopping rule as the serial loop below (a few unused entries may sit
    // between two tables); otherwise the serial loop builds them and refuses
    // PT if they would not fit.
    // The tables hold sum_k len_k entries, and len_k >= min(dmax, 32 ln 2 / db - 2)
    // (below that d, 2^32 exp(-db d) >= exp(2 db) > 1 even after rounding).  When
    // that lower bound passes 2^28 PT is refused without evaluating anything:
    // the same tables the serial loop below ends with.
    {
        long long lower = 0;
        for (int k = 0; k + 1 < R && lower <= (1LL << 28); ++k) {
            const double est = 22.18070977791825 / (betas[k + 1] - betas[k]) - 2.0;
            lower += std::min<long long>(dmax, est > 1.0 ? (long long)std::min(est, 1e18) : 1LL);
        }
        if (lower > (1LL << 28)) {
            out->pt_ok = false;
            swthr.assign(1, 0u);
            return out;
        }
    }
    std::vector<long long> swcap(std::max(R - 1, 1), 0);
    long long bound = 0;
    for (int k = 0; k + 1 < R && bound <= (1LL << 28); ++k) {
        swcap[k] = 1 + std::min<long long>(dmax - 1, (long long)(22.18070977791825 / (betas[k + 1] - betas[k])) + 2);
        bound += swcap[k];
    }
    int k_serial = 0;  // first pair left to the serial loop
    if (R > 2 && bound <= (1LL << 28)) {
        const int npairs = R - 1;
        swthr.assign(size_t(bound), 0u);
        for (int k = 1; k < npairs; ++k)
            swoff[k] = swoff[k - 1] + swcap[k - 1];
        // pairs taken from a shared counter (their tables differ in length)
        const int nthr = std::min(host_threads(), npairs);
        std::atomic<int> next{0};
        host_parallel(nthr, [&](int) {
            for (int k; (k = next.fetch_add(1)) < npairs;) {
                const double db = betas[k + 1] - betas[k];
                uint32_t* v = swthr.data() + swoff[k];  // v[0] = 0: d = 0 never uses the table
                long long d = 1;
                for (; d < dmax && d < swcap[k]; ++d) {
                    const double x = std::floor(std::ldexp(std::exp(-db * double(d)), 32));
                    if (x == 0.0)
                        break;
                    v[d] = uint32_t(x);
                }
                swlen[k] = int(d);
            }
        });
        k_serial = npairs;
    }
    for (int k = k_serial; k + 1 < R; ++k) {
        const double db = betas[k + 1] - betas[k];
        swoff[k] = (long long)swthr.size();
        swthr.push_back(0u);
        long long d = 1;
        for (; d < dmax; ++d) {
            const double v = std::floor(std::ldexp(std::exp(-db * double(d)), 32));
            if (v == 0.0)
                break;
            swthr.push_back(uint32_t(v));
            if (swthr.size() > (size_t(1) << 28))
                break;
        }
        swlen[k] = int(d);
        if (swthr.size() > (size_t(1) << 28)) {
            // a long, finely spaced ladder: the FP64 tables would exceed 2^28
            // entries; sweeps stay available, PT passes are refused
            out->pt_ok = false;
            swthr.assign(1, 0u);
            std::fill(swoff.begin(), swoff.end(), 0LL);
            std::fill(swlen.begin(), swlen.end(), 1);
            break;
        }
    }
    return out;
}

// The tables of the last few ladders (exact betas and bound): handles made
// again and again for the same ladder (a bench loop, a restart, many
// instances of one problem) reuse them instead of evaluating up to millions
// of exponentials each time.  At most kSwapCacheKeep ladders of at most
// 2^24 entries are kept; ising_release_cached_memory empties the cache.
constexpr size_t kSwapCacheKeep = 2;
std::mutex g_swap_mu;
std::vector<std::pair<std::pair<std::vector<double>, long long>, std::shared_ptr<const SwapTables>>> g_swap_cache;

std::shared_ptr<const SwapTables> swap_tables(const double* betas, int R, long long dmax)
{
    std::pair<std::vector<double>, long long> key(std::vector<double>(betas, betas + R), dmax);
    {
        std::lock_guard<std::mutex> lk(g_swap_mu);
        for (size_t i = 0; i < g_swap_cache.size(); ++i)
            if (g_swap_cache[i].first.second == dmax && g_swap_cache[i].first.first.size() == size_t(R) &&
                std::memcmp(g_swap_cache[i].first.first.data(), betas, sizeof(double) * size_t(R)) == 0) {
                auto hit = g_swap_cache[i];
                g_swap_cache.erase(g_swap_cache.begin() + long(i));
                g_swap_cache.push_back(hit);  // most recent last
                return hit.second;
            }
    }
    std::shared_ptr<const SwapTables> t = build_swap_tables(betas, R, dmax);
    if (t->thr.size() <= (size_t(1) << 24)) {
        std::lock_guard<std::mutex> lk(g_swap_mu);
        if (g_swap_cache.size() >= kSwapCacheKeep)
            g_swap_cache.erase(g_swap_cache.begin());
        g_swap_cache.emplace_back(std::move(key), t);
    }
    return t;
}

void swap_cache_clear()
{
    std::lock_guard<std::mutex> lk(g_swap_mu);
    g_swap_cache.clear();
}

}  // namespace

extern "C" {

const char* ising_last_error(void) { return g_err.c_str(); }

int32_t ising_set_alloc_cap(uint64_t bytes)
{
    g_alloc_cap.store(bytes);
    return ISING_OK;
}

int32_t ising_release_cached_memory(void)
{
    big_release_all();
    swap_cache_clear();
    return ISING_OK;
}

int32_t ising_create(int32_t n, const int32_t* row_ptr, const int32_t* col, const int32_t* J,
                     const int32_t* h, int32_t n_slices, uint32_t flags, ising_t* out)
{
    if (!out)
        return fail(ISING_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > (1 << 24))
        return fail(ISING_ERR_INVALID_ARG, "n must be in [1, 2^24]");
    if (!row_ptr || !h || (row_ptr[n] > 0 && (!col || !J)))
        return fail(ISING_ERR_INVALID_ARG, "NULL array");
    if (n_slices < 1 || n % n_slices != 0)
        return fail(ISING_ERR_INVALID_ARG, "n_slices must be >= 1 and divide n");
    if (flags != 0)
        return fail(ISING_ERR_INVALID_ARG, "flags must be 0");
    long long km = 0, eb = 0;
    int32_t rc = validate_csr(n, row_ptr, col, J, h, &km, &eb);
    if (rc)
        return rc;

    ising_s* g = new ising_s();
    g->n = n;
    g->M = n_slices;
    g->S = n / n_slices;
    g->W = (g->M + 31) / 32;
    g->Mp = ((g->M + 3) / 4) * 4;
    const int nnz = row_ptr[n];
    g->row_ptr.assign(row_ptr, row_ptr + n + 1);
    g->col.assign(col, col + nnz);
    g->J.assign(J, J + nnz);
    g->h.assign(h, h + n);
    if (g->S > 65536) {
        delete g;
        return fail(ISING_ERR_UNSUPPORTED, "slice larger than 65536 spins");
    }
    rc = extract_slices(g);
    if (rc) {
        delete g;
        return rc;
    }
    g->kmax = km;
    g->ebound = eb;
    if (eb > (1LL << 30)) {
        delete g;
        return fail(ISING_ERR_FIELD_OVERFLOW, "sum |h| + sum |J| exceeds 2^30");
    }
    cudaError_t ce = device_setup();
    if (ce != cudaSuccess) {
        delete g;
        return cuda_fail(ce, "device setup");
    }
    if ((rc = upload(&g->d_row_ptr, g->row_ptr)) || (rc = upload(&g->d_col, g->col)) ||
        (rc = upload(&g->d_J, g->J)) || (rc = upload(&g->d_h, g->h)) ||
        (rc = upload(&g->d_nbr_off, g->nbr_off)) || (rc = upload(&g->d_nbr, g->nbr)) ||
        (rc = upload(&g->d_jtau, g->jtau)) || (rc = upload(&g->d_lev0, g->lev0p)) ||
        (rc = upload(&g->d_site, g->site)) || (rc = upload(&g->d_pos, g->pos)) ||
        (rc = upload(&g->d_track_off, g->track_off_v)) || (rc = upload(&g->d_track_col, g->track_col))) {
        g->free_all();
        delete g;
        return rc;
    }
    *out = g;
    return ISING_OK;
}

int32_t ising_set_stream(ising_t g, void* s)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (g->stream != static_cast<cudaStream_t>(s))
        g->drop_graphs();
    g->stream = static_cast<cudaStream_t>(s);
    return ISING_OK;
}

// The approximate exponentials of the paper's section 2.4 in FP32 steps: the
// integer n (round half even) plus 127 * 2^23, read as a float, interpolates
// 2^y linearly between integer y; fast: n = round(2^23 x log2 e), scaled by
// 2 ln^2 2; accurate: n = round(2^25 x log2 e) (2^(4y)), scaled, then the
// fourth root as two correctly rounded square roots.
static float approx_exp(float x, bool accurate)
{
    const double ln2 = 0.69314718055994530942, log2e = 1.44269504088896340736;
    const float two_ln2_sq = float(2.0 * ln2 * ln2);
    if (x < float((accurate ? -31.5 : -126.0) * ln2))
        return 0.0f;
    const float a = x * float((accurate ? 33554432.0 : 8388608.0) * log2e);
    const uint32_t bits = uint32_t(int32_t(std::lrint(a)) + 0x3F800000);
    float f;
    std::memcpy(&f, &bits, sizeof f);
    const float e = f * two_ln2_sq;
    return accurate ? std::sqrt(std::sqrt(e)) : e;
}

// T_beta(k) = floor(2^32 min(1, exp(-2 beta k))) in the acceptance mode,
// at most 2^32 - 1
static uint32_t flip_threshold(double beta, long long k, int mode)
{
    if (mode == ISING_ACCEPT_EXACT)
        return uint32_t(std::floor(std::ldexp(std::exp(-2.0 * beta * double(k)), 32)));
    const float e = approx_exp(float(-2.0 * beta * double(k)), mode == ISING_ACCEPT_ACCURATE);
    const double t = std::floor(std::ldexp(double(e), 32));
    return t >= 4294967295.0 ? 0xFFFFFFFFu : uint32_t(t);
}

static int32_t replicas_init_impl(ising_t g, int32_t R, const double* betas, uint32_t seed,
                                  int32_t rng_mode, int32_t field_bits, uint32_t inst);

int32_t ising_set_acceptance(ising_t g, int32_t mode)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (mode != ISING_ACCEPT_EXACT && mode != ISING_ACCEPT_FAST && mode != ISING_ACCEPT_ACCURATE)
        return fail(ISING_ERR_INVALID_ARG, "unknown acceptance mode");
    g->accept_mode = mode;
    return ISING_OK;
}

int32_t ising_replicas_init(ising_t g, int32_t R, const double* betas, uint32_t seed,
                            int32_t rng_mode, int32_t field_bits)
{
    return replicas_init_impl(g, R, betas, seed, rng_mode, field_bits, 0u);
}

static int32_t replicas_init_impl(ising_t g, int32_t R, const double* betas, uint32_t seed,
                                  int32_t rng_mode, int32_t field_bits, uint32_t inst)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (R < 1 || R > (1 << 20) || !betas)
        return fail(ISING_ERR_INVALID_ARG, "R must be in [1, 2^20] with betas given");
    for (int k = 0; k < R; ++k) {
        if (!(betas[k] > 0.0) || !std::isfinite(betas[k]))
            return fail(ISING_ERR_INVALID_ARG, "betas must be finite and > 0");
        if (k > 0 && !(betas[k] > betas[k - 1]))
            return fail(ISING_ERR_INVALID_ARG, "betas must be strictly ascending");
    }
    if (rng_mode != ISING_RNG_MT19937 && rng_mode != ISING_RNG_PHILOX)
        return fail(ISING_ERR_INVALID_ARG, "unknown rng_mode");
    if (field_bits != 16 && field_bits != 32)
        return fail(ISING_ERR_INVALID_ARG, "field_bits must be 16 or 32");
    if (field_bits == 16 && g->kmax > 32767)
        return fail(ISING_ERR_FIELD_OVERFLOW, "max |h_i| + sum_j |J_ij| exceeds int16");
    if ((long long)R * g->n > (1LL << 36))
        return fail(ISING_ERR_INVALID_ARG, "R * n too large");
    g->free_replicas();
    g->learned_passes = 0;
    g->pt_ok = true;
    g->inst = inst;
    g->R = R;
    g->rng = rng_mode;
    g->field_bits = field_bits;
    g->seed = seed;
    g->betas.assign(betas, betas + R);
    g->maxpairs = R / 2;

    // flip thresholds T_beta(k) = floor(2^32 exp(-2 beta k)), FP64 (or the
    // approximate exponential of the handle's acceptance mode); k >= K -> 0
    const int amode = g->accept_mode;
    long long kz = g->kmax + 1;
    for (long long k = 1; k <= g->kmax; ++k)
        if (flip_threshold(betas[0], k, amode) == 0u) {
            kz = k;
            break;
        }
    g->K = int(std::max<long long>(1, std::min<long long>(g->kmax + 1, kz)));
    std::vector<uint32_t> thr(size_t(R) * g->K, 0u);
    for (int t = 0; t < R; ++t)
        for (int k = 1; k < g->K; ++k)
            thr[size_t(t) * g->K + k] = flip_threshold(betas[t], k, amode);
    // swap thresholds of the ladder (shared with earlier handles of the same ladder)
    const std::shared_ptr<const SwapTables> swt = swap_tables(betas, R, 2 * g->ebound + 1);
    g->pt_ok = swt->pt_ok;
    const std::vector<uint32_t>& swthr = swt->thr;
    const std::vector<long long>& swoff = swt->off;
    const std::vector<int>& swlen = swt->len;
    int32_t rc;
    const size_t RN = size_t(R) * g->n;
    if ((rc = dalloc(&g->d_spins, RN)))
        return rc;
    {
        const size_t fbytes = ((RN * (field_bits / 8)) + 15) & ~size_t(15);
        if (!alloc_allowed(fbytes))
            return fail(ISING_ERR_OOM, "device allocation of " + std::to_string(fbytes) + " bytes exceeds the cap");
        cudaError_t e = cudaMalloc(&g->d_fields, fbytes);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMalloc fields");
    }
    std::vector<int> ident(R);
    for (int r = 0; r < R; ++r)
        ident[r] = r;
    if ((rc = dalloc(&g->d_E, R)) || (rc = upload(&g->d_temp, ident)) ||
        (rc = upload(&g->d_slot, ident)) || (rc = dalloc(&g->d_err, 1)) ||
        (rc = dalloc(&g->d_swap_acc, std::max(R - 1, 1))) || (rc = dalloc(&g->d_counters, 2)) ||
        (rc = dalloc(&g->d_done, 1)) || (rc = upload(&g->d_thr, thr)) ||
        (rc = upload(&g->d_swthr, swthr)) || (rc = upload(&g->d_swoff, swoff)) ||
        (rc = upload(&g->d_swlen, swlen)) || (rc = dalloc(&g->d_Epub, 2 * size_t(R))) ||
        (rc = upload(&g->d_betas, g->betas)) ||
        (rc = upload(&g->d_betas32, std::vector<float>(g->betas.begin(), g->betas.end()))) ||
        (rc = dalloc(&g->d_gridbar, 1))) {
        g->free_replicas();
        return rc;
    }
    if (rng_mode == ISING_RNG_MT19937) {
        std::vector<uint32_t> ring(size_t(R + 1) * kMtRing);
        std::vector<unsigned long long> pos(R + 1, 624ull);
        const int nthr = R >= 64 ? std::min(host_threads(), R + 1) : 1;
        host_parallel(nthr, [&](int p) {
            for (int r = p; r <= R; r += nthr)
                mt_seed_ring(seed + uint32_t(r), ring.data() + size_t(r) * kMtRing);
        });
        if ((rc = upload(&g->d_mtring, ring)) || (rc = upload(&g->d_mtpos, pos))) {
            g->free_replicas();
            return rc;
        }
    }
    if ((rc = choose_launch(g))) {
        g->free_replicas();
        return rc;
    }
    // initial spins, fields, energies
    if (rng_mode == ISING_RNG_MT19937) {
        MtGenArgs a{};
        a.ring = g->d_mtring;
        a.pos = g->d_mtpos;
        a.R = R;
        a.mode = 1;
        a.nwords = g->n;
        a.N = g->n;
        a.S = g->S;
        a.M = g->M;
        a.Mp = g->Mp;
        a.spins = g->d_spins;
        a.counters = g->d_counters;
        CK(launch_mt_gen(a, R, g->stream));
    } else {
        CK(launch_philox_init(g->d_spins, R, g->n, g->S, seed, g->inst, g->stream));
    }
    CK(launch_state_init(g->d_spins, g->d_fields, field_bits, g->d_E, R, g->n, g->d_row_ptr,
                         g->d_col, g->d_J, g->d_h, g->stream));
    // ising_run_noalloc's scratch: its device address is resolved (and its
    // module loaded) here, so that the allocation-free run loads nothing
    if ((rc = isg_noalloc_prepare())) {
        g->free_replicas();
        return rc;
    }
    g->inited = true;
    return ISING_OK;
}

static int32_t run_ops(ising_t g, long long n, int swap_every, bool use_graph)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (g->split && !(g->use_fast && g->use_lean))
        return fail(ISING_ERR_UNSUPPORTED, "split couplings need the lean kernel (this launch configuration has none)");
    const long long cap = (n > 0) ? words_cap(g, n) : 1;
    int32_t rc = ensure_buffers(g, cap, cap);
    if (rc)
        return rc;
    std::vector<Op> ops = plan(g, n, swap_every, cap);
    bool has_fused = false;
    for (const Op& op : ops)
        has_fused |= op.kind == Op::FUSED;
    const auto counts = count_kernels(g, ops);
    g->n_launches += counts.first;
    g->n_sweep_launches += counts.second;
    // persistent runs are one or two launches and profiled runs time each
    // launch: neither needs a graph
    if (!use_graph || has_fused || g->profiling)
        return enqueue(g, ops, g->stream);
    const auto key = std::make_pair(n, swap_every);
    auto it = g->graphs.find(key);
    if (it == g->graphs.end()) {
        // record on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the handle's stream
        if (!g->cap_stream)
            CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        rc = enqueue(g, ops, g->cap_stream);
        cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        if (rc) {
            if (graph)
                cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaGraphInstantiate");
        it = g->graphs.emplace(key, exec).first;
    }
    CK(cudaGraphLaunch(it->second, g->stream));
    return ISING_OK;
}

int32_t ising_sweep(ising_t g, int64_t n)
{
    if (n < 0)
        return fail(ISING_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0)
        return (g && g->inited) ? ISING_OK : fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    return run_ops(g, n, 0, false);
}

int32_t ising_pt_swap(ising_t g)
{
    if (g && g->inited && !g->pt_ok && !g->split)
        return fail(ISING_ERR_UNSUPPORTED, "PT swap tables exceed 2^28 entries for this ladder: sweeps only");
    return run_ops(g, 0, -1, false);
}

int32_t ising_run(ising_t g, int64_t n, int32_t swap_every)
{
    if (n < 0)
        return fail(ISING_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0)
        return (g && g->inited) ? ISING_OK : fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    if (g && g->inited && swap_every > 0 && swap_every <= n && !g->pt_ok && !g->split)
        return fail(ISING_ERR_UNSUPPORTED, "PT swap tables exceed 2^28 entries for this ladder: sweeps only");
    return run_ops(g, n, swap_every > 0 ? swap_every : 0, true);
}

int32_t ising_read_state(ising_t g, int8_t* spins, int32_t* fields, int64_t* energy,
                         int32_t* temp_of_slot, uint64_t* counters)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    int32_t rc = check_device_error(g);
    if (rc)
        return rc;
    const size_t RN = size_t(g->R) * g->n;
    if (spins)
        CK(cudaMemcpyAsync(spins, g->d_spins, RN, cudaMemcpyDeviceToHost, g->stream));
    if (fields) {
        if (g->field_bits == 32) {
            CK(cudaMemcpyAsync(fields, g->d_fields, RN * 4, cudaMemcpyDeviceToHost, g->stream));
        } else {
            // widened on the device in chunks of at most 16 Mi fields (64 MB of
            // scratch), each copied straight into the caller's buffer
            const size_t chunk = std::min<size_t>(RN, size_t(1) << 24);
            if (g->widen_cap < chunk) {
                dfree(g->d_widen);
                g->widen_cap = 0;
                if ((rc = dalloc(&g->d_widen, chunk)))
                    return rc;
                g->widen_cap = chunk;
            }
            const int16_t* src = static_cast<const int16_t*>(g->d_fields);
            for (size_t o = 0; o < RN; o += chunk) {
                const size_t m = std::min(chunk, RN - o);
                CK(launch_widen_i16(src + o, g->d_widen, (long long)m, g->stream));
                CK(cudaMemcpyAsync(fields + o, g->d_widen, m * 4, cudaMemcpyDeviceToHost, g->stream));
            }
        }
    }
    std::vector<int> e32(g->R);
    CK(cudaMemcpyAsync(e32.data(), g->d_E, sizeof(int) * g->R, cudaMemcpyDeviceToHost, g->stream));
    if (temp_of_slot)
        CK(cudaMemcpyAsync(temp_of_slot, g->d_temp, sizeof(int) * g->R, cudaMemcpyDeviceToHost,
                           g->stream));
    unsigned long long cnt[2] = {0, 0};
    CK(cudaMemcpyAsync(cnt, g->d_counters, sizeof(cnt), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (energy)
        for (int r = 0; r < g->R; ++r)
            energy[r] = e32[r];
    if (counters) {
        counters[0] = cnt[0];
        counters[1] = cnt[1];
    }
    return ISING_OK;
}

// Split-coupling flip threshold of temperature beta with Trotter coupling K:
// z = 2 (beta k_s + K k_tau), each product rounded on its own (volatile keeps
// the host compiler from fusing them); T = min(floor(2^32 e^-z), 2^32 - 1),
// 2^32 - 1 for z <= 0 (that value accepts every word).
static uint32_t split_flip_threshold(double beta, double K, int ks, int kt)
{
    volatile double a = beta * double(ks);
    volatile double b = K * double(kt);
    const double z = 2.0 * (a + b);
    if (z <= 0.0)
        return 0xFFFFFFFFu;
    const double t = std::floor(std::ldexp(std::exp(-z), 32));
    return t >= 4294967295.0 ? 0xFFFFFFFFu : uint32_t(t);
}

// Flip tables of R temperatures: entry (k_s + ks) * 3 + k_tau / 2 + 1 of
// temperature t (stride 3 (2 ks + 1)) for k_s in [-ks, ks], k_tau in {-2, 0, 2}.
static void split_flip_table(const double* betas, const double* K, int R, int ks, uint32_t* out)
{
    const size_t Ks = size_t(3) * size_t(2 * ks + 1);
    const int nthr = (double(R) * double(Ks) >= 65536.0) ? std::min(host_threads(), R) : 1;
    isg::host_parallel(nthr, [&](int p) {
        for (int t = p; t < R; t += nthr)
            for (int k = -ks; k <= ks; ++k)
                for (int j = 0; j < 3; ++j)
                    out[size_t(t) * Ks + size_t(k + ks) * 3 + j] =
                        split_flip_threshold(betas[t], K[t], k, 2 * j - 2);
    });
}

int32_t ising_split_flip_table(int32_t R, const double* betas, const double* K, int32_t ks, uint32_t* out)
{
    if (R < 1 || !betas || !K || !out || ks < 0 || ks > 1364)
        return fail(ISING_ERR_INVALID_ARG, "R >= 1, 0 <= ks <= 1364 and non-NULL arrays required");
    split_flip_table(betas, K, R, ks, out);
    return ISING_OK;
}

double ising_split_exp(double x) { return isg::split_detail::exp_det(x); }

int32_t ising_swap_thresholds(int32_t R, const double* betas, int64_t dmax, uint32_t* thr, int64_t cap,
                              int64_t* off, int32_t* len, int64_t* n_entries, int32_t* pt_ok)
{
    if (R < 1 || !betas || dmax < 1 || !n_entries)
        return fail(ISING_ERR_INVALID_ARG, "R >= 1, dmax >= 1, betas and n_entries required");
    for (int k = 1; k < R; ++k)
        if (!(betas[k] > betas[k - 1]))
            return fail(ISING_ERR_INVALID_ARG, "betas must be strictly ascending");
    const std::shared_ptr<const SwapTables> t = build_swap_tables(betas, R, (long long)dmax);
    *n_entries = (int64_t)t->thr.size();
    if (pt_ok)
        *pt_ok = t->pt_ok ? 1 : 0;
    if (off)
        for (int k = 0; k + 1 < R; ++k)
            off[k] = t->off[size_t(k)];
    if (len)
        for (int k = 0; k + 1 < R; ++k)
            len[k] = t->len[size_t(k)];
    if (thr) {
        if (cap < (int64_t)t->thr.size())
            return fail(ISING_ERR_INVALID_ARG, "thr holds fewer than n_entries values");
        std::copy(t->thr.begin(), t->thr.end(), thr);
    }
    return ISING_OK;
}

uint32_t ising_split_swap_threshold(double dbeta, double dK, int64_t dE, int64_t dC)
{
    return isg::split_detail::swap_threshold(dbeta, dK, (long long)dE, (long long)dC);
}

int32_t ising_set_trotter(ising_t g, const double* K)
{
    if (!g || !K)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    const int R = g->R;
    for (int k = 0; k < R; ++k)
        if (!std::isfinite(K[k]))
            return fail(ISING_ERR_INVALID_ARG, "Trotter couplings must be finite");
    if (g->split)
        return fail(ISING_ERR_INVALID_ARG, "split couplings are already set: call ising_replicas_init first");
    if (g->accept_mode != ISING_ACCEPT_EXACT)
        return fail(ISING_ERR_UNSUPPORTED, "split couplings use the exact exponential (ISING_ACCEPT_EXACT)");
    if (g->M < 3 || g->S < 1)
        return fail(ISING_ERR_UNSUPPORTED, "split couplings need declared slices with a Trotter ring (M >= 3)");
    // k_space bound: max_i |h_i| + sum over spatial j of |J_ij| (slices are identical)
    long long ks = 0;
    for (int q = 0; q < g->S; ++q) {
        long long b = std::llabs((long long)g->h[q]);
        for (int e = g->row_ptr[q]; e < g->row_ptr[q + 1]; ++e)
            if (g->col[e] < g->S)
                b += std::llabs((long long)g->J[e]);
        ks = std::max(ks, b);
    }
    const long long Ks = 3 * (2 * ks + 1);
    if (Ks > 8192)
        return fail(ISING_ERR_UNSUPPORTED, "split-coupling flip table exceeds 8192 entries per temperature");
    std::vector<uint32_t> thr(size_t(R) * size_t(Ks));
    split_flip_table(g->betas.data(), K, R, int(ks), thr.data());
    std::vector<double> dbeta(std::max(R - 1, 1), 0.0), dK(std::max(R - 1, 1), 0.0);
    for (int k = 0; k + 1 < R; ++k) {
        dbeta[k] = g->betas[k + 1] - g->betas[k];
        dK[k] = K[k + 1] - K[k];
    }
    // nothing queued may still read the plain tables or fields
    CK(cudaStreamSynchronize(g->stream));
    uint32_t* d_thr = nullptr;
    int *d_C = nullptr, *d_Cpub = nullptr;
    double *d_db = nullptr, *d_dk = nullptr;
    int32_t rc;
    if ((rc = upload(&d_thr, thr)) || (rc = dalloc(&d_C, R)) || (rc = dalloc(&d_Cpub, 2 * size_t(R))) ||
        (rc = upload(&d_db, dbeta)) || (rc = upload(&d_dk, dK))) {
        dfree(d_thr);
        dfree(d_C);
        dfree(d_Cpub);
        dfree(d_db);
        dfree(d_dk);
        return rc;
    }
    const int K_plain = g->K;
    uint32_t* thr_plain = g->d_thr;
    g->split = true;
    g->split_ks = int(ks);
    g->K = int(Ks);
    g->d_thr = d_thr;
    g->drop_graphs();
    rc = choose_launch(g);
    if (rc || !(g->use_fast && g->use_lean)) {
        // no lean launch for this model or configuration: back to plain couplings
        g->split = false;
        g->split_ks = 0;
        g->K = K_plain;
        g->d_thr = thr_plain;
        dfree(d_thr);
        dfree(d_C);
        dfree(d_Cpub);
        dfree(d_db);
        dfree(d_dk);
        const int32_t rc2 = choose_launch(g);
        if (rc2)
            return rc2;
        return fail(ISING_ERR_UNSUPPORTED, "split couplings need the lean kernel, which this model or launch "
                                           "configuration does not allow");
    }
    dfree(thr_plain);
    g->d_C = d_C;
    g->d_Cpub = d_Cpub;
    g->d_dbeta = d_db;
    g->d_dK = d_dk;
    g->trotter_K.assign(K, K + R);
    CK(launch_split_state_init(g->d_spins, g->d_fields, g->field_bits, g->d_E, g->d_C, R, g->n, g->S,
                               g->d_row_ptr, g->d_col, g->d_J, g->d_h, g->stream));
    return ISING_OK;
}

int32_t ising_read_trotter(ising_t g, int64_t* C)
{
    if (!g || !C)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    if (!g->split) {
        std::fill(C, C + g->R, int64_t(0));
        return ISING_OK;
    }
    int32_t rc = check_device_error(g);
    if (rc)
        return rc;
    std::vector<int> c32(g->R);
    CK(cudaMemcpyAsync(c32.data(), g->d_C, sizeof(int) * g->R, cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    for (int r = 0; r < g->R; ++r)
        C[r] = c32[r];
    return ISING_OK;
}

int32_t ising_read_swap_stats(ising_t g, uint64_t* accepted)
{
    if (!g || !accepted)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    if (g->R < 2)
        return ISING_OK;
    CK(cudaMemcpyAsync(accepted, g->d_swap_acc, sizeof(uint64_t) * (g->R - 1),
                       cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return ISING_OK;
}

namespace {
struct BlobHeader {
    uint32_t magic, version;
    int32_t n, R, field_bits, rng, M, pad;
};
constexpr uint32_t kMagic = 0x31475349u;  // "ISG1"

// Version 2: the state, then the generator key {seed, instance} (what Philox
// words depend on; MT19937 streams are in the rings) and the count of learned
// passes (their Philox counter), then with split couplings (bit 0 of `pad`)
// K [R] (FP64) and C [R] (int32).  Version 1 (read only) has neither the key
// nor split couplings.
size_t blob_size_v1(const ising_s* g)
{
    const size_t RN = size_t(g->R) * g->n;
    size_t s = sizeof(BlobHeader) + RN + RN * (g->field_bits / 8) + 4 * size_t(g->R) * 3 +
               8 * size_t(std::max(g->R - 1, 1)) + 16;
    if (g->rng == ISING_RNG_MT19937)
        s += 4 * size_t(g->R + 1) * kMtRing + 8 * size_t(g->R + 1);
    return s;
}

size_t blob_size_for(const ising_s* g, bool split)
{
    return blob_size_v1(g) + 16 + (split ? 12 * size_t(g->R) : 0);
}

size_t blob_size(ising_s* g) { return blob_size_for(g, g->split); }
}  // namespace

int32_t ising_save(ising_t g, void* buf, size_t cap, size_t* size)
{
    if (!g || !size)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    const size_t need = blob_size(g);
    *size = need;
    if (!buf)
        return ISING_OK;
    if (cap < need)
        return fail(ISING_ERR_INVALID_ARG, "buffer too small");
    int32_t rc = check_device_error(g);
    if (rc)
        return rc;
    char* p = static_cast<char*>(buf);
    BlobHeader hd{kMagic, 2u, g->n, g->R, g->field_bits, g->rng, g->M, g->split ? 1 : 0};
    std::memcpy(p, &hd, sizeof hd);
    p += sizeof hd;
    const size_t RN = size_t(g->R) * g->n;
    auto d2h = [&](const void* d, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(p, d, bytes, cudaMemcpyDeviceToHost, g->stream);
        p += bytes;
        return e;
    };
    CK(d2h(g->d_spins, RN));
    CK(d2h(g->d_fields, RN * (g->field_bits / 8)));
    CK(d2h(g->d_E, 4 * size_t(g->R)));
    CK(d2h(g->d_temp, 4 * size_t(g->R)));
    CK(d2h(g->d_slot, 4 * size_t(g->R)));
    CK(d2h(g->d_swap_acc, 8 * size_t(std::max(g->R - 1, 1))));
    CK(d2h(g->d_counters, 16));
    if (g->rng == ISING_RNG_MT19937) {
        CK(d2h(g->d_mtring, 4 * size_t(g->R + 1) * kMtRing));
        CK(d2h(g->d_mtpos, 8 * size_t(g->R + 1)));
    }
    const uint32_t key[2] = {g->seed, g->inst};
    std::memcpy(p, key, sizeof key);
    p += sizeof key;
    const unsigned long long lp = g->learned_passes;
    std::memcpy(p, &lp, sizeof lp);
    p += sizeof lp;
    if (g->split) {
        std::memcpy(p, g->trotter_K.data(), 8 * size_t(g->R));
        p += 8 * size_t(g->R);
        CK(d2h(g->d_C, 4 * size_t(g->R)));
    }
    CK(cudaStreamSynchronize(g->stream));
    return ISING_OK;
}

int32_t ising_load(ising_t g, const void* buf, size_t size)
{
    if (!g || !buf)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "not initialised");
    if (size < sizeof(BlobHeader))
        return fail(ISING_ERR_INVALID_ARG, "blob too small");
    const char* p = static_cast<const char*>(buf);
    BlobHeader hd;
    std::memcpy(&hd, p, sizeof hd);
    p += sizeof hd;
    if (hd.magic != kMagic || (hd.version != 1u && hd.version != 2u))
        return fail(ISING_ERR_INVALID_ARG, "not a checkpoint blob of this library");
    const bool bsplit = hd.version == 2u && (hd.pad & 1);
    if (size != (hd.version == 1u ? blob_size_v1(g) : blob_size_for(g, bsplit)))
        return fail(ISING_ERR_INVALID_ARG, "blob size does not match this handle");
    if (hd.n != g->n || hd.R != g->R || hd.field_bits != g->field_bits || hd.rng != g->rng || hd.M != g->M)
        return fail(ISING_ERR_INVALID_ARG, "blob was saved from a different configuration");
    if (bsplit) {
        // the couplings first: a plain handle takes the blob's split couplings
        std::vector<double> Kb(g->R);
        std::memcpy(Kb.data(), static_cast<const char*>(buf) + blob_size_v1(g) + 16, 8 * size_t(g->R));
        if (g->split) {
            if (std::memcmp(Kb.data(), g->trotter_K.data(), 8 * size_t(g->R)) != 0)
                return fail(ISING_ERR_INVALID_ARG, "blob was saved with other Trotter couplings");
        } else {
            const int32_t rc = ising_set_trotter(g, Kb.data());
            if (rc)
                return rc;
        }
    } else if (g->split) {
        return fail(ISING_ERR_INVALID_ARG, "blob holds plain couplings; this handle has split couplings");
    }
    const size_t RN = size_t(g->R) * g->n;
    auto h2d = [&](void* d, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, g->stream);
        p += bytes;
        return e;
    };
    CK(h2d(g->d_spins, RN));
    CK(h2d(g->d_fields, RN * (g->field_bits / 8)));
    CK(h2d(g->d_E, 4 * size_t(g->R)));
    CK(h2d(g->d_temp, 4 * size_t(g->R)));
    CK(h2d(g->d_slot, 4 * size_t(g->R)));
    CK(h2d(g->d_swap_acc, 8 * size_t(std::max(g->R - 1, 1))));
    CK(h2d(g->d_counters, 16));
    if (g->rng == ISING_RNG_MT19937) {
        CK(h2d(g->d_mtring, 4 * size_t(g->R + 1) * kMtRing));
        CK(h2d(g->d_mtpos, 8 * size_t(g->R + 1)));
    }
    if (hd.version >= 2u) {
        uint32_t key[2];
        std::memcpy(key, p, sizeof key);
        p += sizeof key;
        g->seed = key[0];  // Philox words of later sweeps follow the saved key
        g->inst = key[1];
        unsigned long long lp;
        std::memcpy(&lp, p, sizeof lp);
        p += sizeof lp;
        g->learned_passes = lp;
        g->drop_graphs();  // recorded launches hold the old key
    }
    if (bsplit) {
        p += 8 * size_t(g->R);  // K, applied above
        CK(h2d(g->d_C, 4 * size_t(g->R)));
    }
    CK(cudaStreamSynchronize(g->stream));
    return ISING_OK;
}

int32_t ising_set_seed(ising_t g, uint32_t seed)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (!g->inited)
        return fail(ISING_ERR_NOT_INITIALISED, "call ising_replicas_init first");
    if (g->rng != ISING_RNG_PHILOX)
        return fail(ISING_ERR_UNSUPPORTED, "ising_set_seed needs ISING_RNG_PHILOX");
    g->seed = seed;
    g->drop_graphs();  // recorded launches hold the old key
    return ISING_OK;
}

int32_t ising_get_info(ising_t g, ising_info_t* o)
{
    if (!g || !o)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    std::memset(o, 0, sizeof *o);
    o->n = g->n;
    o->slices = g->M;
    o->slice_size = g->S;
    o->levels = g->D;
    o->slice_depth = g->D0;
    o->replicas = g->R;
    o->replicas_per_block = g->G;
    o->threads_per_block = g->T;
    o->blocks = g->blocks;
    o->smem_bytes = int(g->smem);
    o->persistent_ok = g->persistent_ok ? 1 : 0;
    o->fast_kernel = g->use_fast ? (g->use_packed ? 4 : (g->use_track ? 3 : (g->use_lean ? 2 : 1))) : 0;
    o->field_bits = g->field_bits;
    o->rng_mode = g->rng;
    o->kmax = int(std::min<long long>(g->kmax, INT32_MAX));
    return ISING_OK;
}

int32_t ising_set_launch(ising_t g, int32_t replicas_per_block, int32_t threads_per_block,
                         int32_t launch_flags)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    if (replicas_per_block < 0 || (replicas_per_block & (replicas_per_block - 1)) ||
        replicas_per_block > 32)
        return fail(ISING_ERR_INVALID_ARG, "replicas_per_block must be 0 or a power of two <= 32");
    g->G_req = replicas_per_block;
    g->T_req = threads_per_block;
    g->allow_persistent = (launch_flags & ISING_LAUNCH_PERSISTENT) ? 1 : 0;
    g->fast_off = (launch_flags & ISING_LAUNCH_GENERIC) != 0;
    g->lean_off = (launch_flags & ISING_LAUNCH_NO_LEAN) != 0;
    g->track_on = (launch_flags & ISING_LAUNCH_TRACK) != 0;
    g->packed_off = (launch_flags & ISING_LAUNCH_NO_PACKED) != 0;
    g->drop_graphs();
    if (g->inited)
        return choose_launch(g);
    return ISING_OK;
}

int32_t ising_set_profiling(ising_t g, int32_t on)
{
    if (!g)
        return fail(ISING_ERR_INVALID_ARG, "NULL handle");
    g->profiling = on != 0;
    return ISING_OK;
}

int32_t ising_get_stats(ising_t g, ising_stats_t* out)
{
    if (!g || !out)
        return fail(ISING_ERR_INVALID_ARG, "NULL argument");
    if (!g->ev_pending.empty()) {
        CK(cudaStreamSynchronize(g->stream));
        for (auto& ev : g->ev_pending) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ev.first, ev.second));
            g->kernel_ms += ms;
            ++g->n_timed;
            cudaEventDestroy(ev.first);
            cudaEventDestroy(ev.second);
        }
        g->ev_pending.clear();
    }
    out->launches = g->n_launches;
    out->sweep_launches = g->n_sweep_launches;
    out->timed_launches = g->n_timed;
    out->kernel_ms = g->kernel_ms;
    return ISING_OK;
}

int32_t ising_destroy(ising_t g)
{
    if (!g)
        return ISING_OK;
    g->free_all();
    delete g;
    return ISING_OK;
}

}  // extern "C"

// ============================================================ ragged batches
// A batch owns one ordinary handle per instance.  Instances are grouped by
// launch shape (kernel variant, field width, generator, columns per thread,
// threads per block); every planned op of a group becomes ONE batched launch
// whose blocks are (instance, block) items, and the groups run as parallel
// branches of one recorded CUDA graph.
struct PackedWave {
    int T = 0;               // sweep threads per block (every instance of the wave)
    int rmax = 1;            // slot rounds per thread
    size_t smem = 0;         // dynamic shared memory: the largest instance's
    std::vector<int> ids;    // instances, longest level count first
    long long blocks = 0;    // replicas of the wave (one block each)
};

struct ising_batch_s {
    std::vector<ising_s*> inst;
    std::vector<int> resident;  // 1: the whole ladder runs as one block
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to record graphs
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    struct Run {
        cudaGraphExec_t exec = nullptr;
        std::vector<void*> bufs;  // device argument records of the graph
        // persistent (packed) batches: the launches of a call, each one wave
        // for `sweeps` sweeps with PT every `every` (0: none)
        struct Launch {
            int wave, sweeps, every, n_items;
            const SweepArgs* args;
            const BatchItem* items;
            const MtGenArgs* gen;  // MT19937: the wave's swap-stream words (or null)
            const BatchItem* gen_items;
            int n_gen;
        };
        std::vector<Launch> launches;
        bool no_graph = false;  // recording was refused: launched directly
    };
    std::map<std::pair<long long, int>, Run> runs;
    // persistent batches of the packed kernel (waves of whole, co-resident instances)
    bool packed = false;
    std::vector<PackedWave> waves;
    unsigned* d_bar = nullptr;  // [instances] grid-barrier counters of the persistent launches

    void drop_runs()
    {
        for (auto& kv : runs) {
            if (kv.second.exec)
                cudaGraphExecDestroy(kv.second.exec);
            for (void* p : kv.second.bufs)
                cudaFree(p);
        }
        runs.clear();
    }
};

namespace {

constexpr int kBatchSide = 32;  // parallel graph branches

struct GroupKey {
    int kind;  // 0 resident (fused PT in one block), 1 streamed, 2 generic kernel
    int lean, field_bits, rng, cmax, T;
    bool operator<(const GroupKey& o) const
    {
        return std::tie(kind, lean, field_bits, rng, cmax, T) <
               std::tie(o.kind, o.lean, o.field_bits, o.rng, o.cmax, o.T);
    }
};

int pow2_at_least(int x)
{
    int p = 1;
    while (p < x)
        p <<= 1;
    return p;
}

// Launch shape of an instance: `resident` asks for the whole ladder in one
// block (G = next power of two >= R) with `T` threads (0 = automatic); else
// the default shape without the persistent launch.  Returns whether the
// instance ended up resident.
bool configure_instance(ising_s* g, bool resident, int T, int G_streamed = 0)
{
    if (resident) {
        const int G = pow2_at_least(g->R);
        int Tr = T;
        if (Tr <= 0) {
            // fewest columns per thread that the thread cap allows
            const long long cols = (long long)g->S * G;
            for (int cm : {2, 4, 8}) {
                const int tmax = cm <= 2 ? 1024 : (cm == 4 ? 512 : 256);
                const int step = std::max(32, G);
                const long long t = ((cols + cm - 1) / cm + step - 1) / step * step;
                if (t <= tmax) {
                    Tr = int(std::max<long long>(t, step));
                    break;
                }
            }
        }
        if (G <= 64 && Tr > 0 && Tr <= 1024 && Tr % G == 0) {
            g->G_req = G;
            g->T_req = Tr;
            g->allow_persistent = 1;
            if (choose_launch(g) == ISING_OK && g->use_fast && g->blocks == 1 && g->persistent_ok)
                return true;
        }
    }
    g->G_req = G_streamed;
    g->T_req = resident ? 0 : T;
    g->allow_persistent = 0;
    if (choose_launch(g) != ISING_OK) {
        g->G_req = 0;
        g->T_req = 0;
        choose_launch(g);
    }
    return false;
}

GroupKey key_of(ising_batch_s* b, int i)
{
    ising_s* g = b->inst[i];
    GroupKey k{};
    k.kind = b->resident[i] ? 0 : (g->use_fast ? 1 : 2);
    k.lean = kernel_variant(g);
    k.field_bits = g->field_bits;
    k.rng = g->rng;
    k.cmax = g->use_fast ? g->fast_cmax : g->cmax;
    k.T = g->T;
    return k;
}

template <typename T>
int32_t upload_raw(std::vector<void*>& keep, const std::vector<T>& h, const T** out)
{
    T* d = nullptr;
    int32_t rc = dalloc(&d, std::max<size_t>(h.size(), 1));
    if (rc)
        return rc;
    keep.push_back(d);
    if (!h.empty())
        CK(cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = d;
    return ISING_OK;
}

}  // namespace

namespace {

// A group's ops, each with the device argument records of its batched launch.
struct BatchOp {
    Op op;
    const void* args = nullptr;      // MtGenArgs / SweepArgs / PtArgs per instance
    const BatchItem* items = nullptr;
    int n_items = 0;
};

struct BatchGroup {
    GroupKey key;
    std::vector<int> ids;
    std::vector<BatchOp> ops;
    size_t smem_plain = 0, smem_fused = 0;
    int max_S = 0, max_R = 0;
};

// ---------------------------------------------- persistent packed batches
// Instances whose models the packed kernel takes run as waves: whole
// instances whose replicas (one block each) are resident together, grouped
// by block shape and ordered by level count, one cooperative launch per wave
// for all sweeps of a call with every instance's PT passes fused behind its
// own bounded barrier.  Returns whether the batch runs this way.
bool packed_batch_setup(ising_batch_s* b)
{
    if (!g_coop)
        return false;
    const int gen = kPackedGenWarps;  // the generator warps (both generators)
    std::map<std::pair<int, int>, std::vector<int>> by_T;  // (sweep threads, rounds)
    const int n_inst = int(b->inst.size());
    std::vector<size_t> smem(n_inst, 0);
    // one slot per thread up to 256 slots, else 128 threads of three rounds
    auto threads_of = [](const ising_s* g) { return g->nslots <= 256 ? ((g->nslots + 31) / 32) * 32 : 128; };
    for (const ising_s* g : b->inst) {
        const bool ok = (g->M == 8 || g->M == 16 || g->M == 32) && g->max_sp_deg <= 6 && g->max_sp_J <= 127 &&
                        g->S < 65536 && g->D0 < 65536 && g->nslots >= 1 && g->nslots <= 384 && !g->split &&
                        g->R <= 16384;
        if (!ok)
            return false;
    }
    // the instances' tables (with their word placement searches) on the host
    // threads, then uploaded in order
    std::vector<std::vector<uint32_t>> pks(n_inst);
    {
        const int nthr = std::max(1, std::min(isg::host_threads(), n_inst));
        isg::host_parallel(nthr, [&](int p) {
            for (int i = p; i < n_inst; i += nthr)
                if (!b->inst[i]->d_pk)
                    pks[i] = packed_tables(b->inst[i], threads_of(b->inst[i]));
        });
    }
    for (int i = 0; i < n_inst; ++i) {
        ising_s* g = b->inst[i];
        const int T = threads_of(g);
        if (!g->d_pk) {
            if (upload(&g->d_pk, pks[i]) != ISING_OK)
                return false;
            g->pk_bytes = uint32_t(pks[i].size() * 4);
            std::vector<uint32_t>().swap(pks[i]);
        }
        const int rmax = g->nslots <= 256 ? 1 : 3;
        SweepArgs a = base_args(g);
        a.G = 1;
        a.gen = gen;
        a.swap_every = 1;
        smem[i] = packed_smem_bytes(a, T);
        by_T[std::make_pair(T, rmax)].push_back(i);
    }
    const size_t lim = sweep_max_dynamic_smem() ? sweep_max_dynamic_smem() : 200 * 1024;
    std::vector<PackedWave> waves;
    for (auto& kv : by_T) {
        const int T = kv.first.first, rmax = kv.first.second;
        std::vector<int>& ids = kv.second;
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return b->inst[x]->D > b->inst[y]->D; });
        PackedWave w;
        w.T = T;
        w.rmax = rmax;
        long long cap = 0;
        for (int i : ids) {
            const size_t sm = std::max(w.smem, smem[i]);
            int per_sm = 0;
            if (sm > lim || fast_max_blocks_per_sm_batch(b->inst[i]->rng, rmax, T + 32 * gen, sm, &per_sm) != cudaSuccess)
                return false;
            cap = (long long)per_sm * g_num_sms;
            if (!w.ids.empty() && w.blocks + b->inst[i]->R > cap) {
                waves.push_back(w);
                w = PackedWave{};
                w.T = T;
                w.rmax = rmax;
                if (fast_max_blocks_per_sm_batch(b->inst[i]->rng, rmax, T + 32 * gen, smem[i], &per_sm) != cudaSuccess)
                    return false;
                cap = (long long)per_sm * g_num_sms;
            }
            if (b->inst[i]->R > cap)
                return false;  // one instance alone is not resident
            w.ids.push_back(i);
            w.smem = std::max(w.smem, smem[i]);
            w.blocks += b->inst[i]->R;
        }
        if (!w.ids.empty())
            waves.push_back(w);
    }
    if (dalloc(&b->d_bar, std::max<size_t>(b->inst.size(), 1)) != ISING_OK)
        return false;
    b->waves = waves;
    return true;
}

// The launches of ising_batch_run(n, swap_every) on a persistent batch:
// every wave for its fused part (whole groups of swap_every sweeps, PT after
// each) and its remainder (no PT), as plan() splits a single instance's run.
int32_t packed_batch_build(ising_batch_s* b, long long n, int swap_every, ising_batch_s::Run* run)
{
    const long long every = swap_every > 0 ? swap_every : 0;
    const long long fused = (every > 0 && n >= every) ? (n / every) * every : 0;
    const long long rest = n - fused;
    const bool mt = b->inst[0]->rng == ISING_RNG_MT19937;
    if (fused > (1LL << 30) || rest > (1LL << 30))
        return fail(ISING_ERR_INVALID_ARG, "a persistent batch run takes at most 2^30 sweeps per call");
    for (int wi = 0; wi < int(b->waves.size()); ++wi) {
        const PackedWave& w = b->waves[wi];
        for (int part = 0; part < 2; ++part) {
            const long long m = part == 0 ? fused : rest;
            if (m == 0)
                continue;
            const int passes = part == 0 ? int(m / every) : 0;
            std::vector<SweepArgs> args;
            std::vector<BatchItem> items;
            std::vector<MtGenArgs> gargs;
            std::vector<BatchItem> gitems;
            int max_S = 0;
            for (int j = 0; j < int(w.ids.size()); ++j) {
                ising_s* g = b->inst[w.ids[j]];
                if (g->wbuf_cap < 2) {  // the sweep kernel's two-sweep word buffer
                    big_free(g->d_wbuf);
                    int32_t rc = big_alloc(&g->d_wbuf, size_t(2) * g->R * g->S * g->Mp);
                    if (rc)
                        return rc;
                    g->wbuf_cap = 2;
                }
                if (mt) {  // the swap stream's words
                    if (passes > g->swbuf_cap) {
                        dfree(g->d_swbuf);
                        int32_t rc = dalloc(&g->d_swbuf, size_t(passes) * std::max(g->maxpairs, 1));
                        if (rc)
                            return rc;
                        g->swbuf_cap = passes;
                    }
                    if (passes > 0) {
                        int blocks = 0;
                        gargs.push_back(gen_args(g, Op{Op::GEN, 0, passes, 0}, &blocks));
                        gitems.push_back({int(gargs.size()) - 1, g->R});
                        max_S = std::max(max_S, g->S);
                    }
                }
                SweepArgs a = base_args(g);
                a.G = 1;
                a.nsweeps = int(m);
                a.swap_every = part == 0 ? int(every) : 0;
                a.inst_blocks = g->R;
                a.sweep_threads = w.T;
                a.gen = kPackedGenWarps;
                a.wbuf = g->d_wbuf;
                a.swbuf = g->d_swbuf;
                a.gridbar = b->d_bar + w.ids[j];
                args.push_back(a);
                for (int k = 0; k < g->R; ++k)
                    items.push_back({j, k});
            }
            ising_batch_s::Run::Launch L{};
            L.wave = wi;
            L.sweeps = int(m);
            L.every = part == 0 ? int(every) : 0;
            L.n_items = int(items.size());
            int32_t rc = upload_raw(run->bufs, args, &L.args);
            if (!rc)
                rc = upload_raw(run->bufs, items, &L.items);
            if (!rc && !gargs.empty()) {
                rc = upload_raw(run->bufs, gargs, &L.gen);
                if (!rc)
                    rc = upload_raw(run->bufs, gitems, &L.gen_items);
                L.n_gen = int(gitems.size());
            }
            if (rc)
                return rc;
            (void)max_S;
            run->launches.push_back(L);
        }
    }
    return ISING_OK;
}

int32_t packed_batch_enqueue(ising_batch_s* b, const ising_batch_s::Run& run, cudaStream_t st)
{
    const bool mt = b->inst[0]->rng == ISING_RNG_MT19937;
    for (const auto& L : run.launches) {
        const PackedWave& w = b->waves[L.wave];
        cudaError_t e = cudaSuccess;
        if (L.n_gen > 0) {
            int max_S = 0;
            for (int i : w.ids)
                max_S = std::max(max_S, b->inst[i]->S);
            e = launch_mt_gen_batch(L.gen, L.gen_items, L.n_gen, max_S, st);
        }
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * b->inst.size(), st);
        if (e == cudaSuccess)
            e = launch_packed_batch(L.args, L.items, L.n_items, mt ? 0 : 1, w.rmax, w.T + 32 * kPackedGenWarps,
                                    w.smem, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "persistent batch launch");
    }
    return ISING_OK;
}

// A call's launches, waves one after another, recorded once into a CUDA
// graph (on the batch's private capture stream) and replayed; if recording
// is refused the launches are enqueued directly.
int32_t packed_batch_launch(ising_batch_s* b, ising_batch_s::Run& run)
{
    if (!run.exec && !run.no_graph) {
        if (!b->cap)
            CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        int32_t rc = e == cudaSuccess ? packed_batch_enqueue(b, run, b->cap) : ISING_OK;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(b->cap, &graph) : e;
        if (!rc && e2 == cudaSuccess && graph && cudaGraphInstantiate(&run.exec, graph, 0) != cudaSuccess)
            run.exec = nullptr;
        if (graph)
            cudaGraphDestroy(graph);
        cudaGetLastError();  // a refused capture leaves no sticky state
        if (!run.exec)
            run.no_graph = true;
    }
    if (run.exec)
        CK(cudaGraphLaunch(run.exec, b->stream));
    else if (int32_t rc = packed_batch_enqueue(b, run, b->stream))
        return rc;
    for (const auto& L : run.launches)
        for (int i : b->waves[L.wave].ids) {
            b->inst[i]->n_launches += 1 + (L.n_gen > 0 ? 1 : 0);
            b->inst[i]->n_sweep_launches += 1;
        }
    return ISING_OK;
}

int32_t batch_record(ising_batch_s* b, long long n, int swap_every, ising_batch_s::Run* run)
{
    std::map<GroupKey, BatchGroup> groups;
    for (int i = 0; i < int(b->inst.size()); ++i) {
        const GroupKey k = key_of(b, i);
        BatchGroup& gr = groups[k];
        gr.key = k;
        gr.ids.push_back(i);
    }
    std::vector<BatchGroup*> order;
    for (auto& kv : groups) {
        BatchGroup& gr = kv.second;
        order.push_back(&gr);
        long long cap = LLONG_MAX;
        for (int i : gr.ids) {
            ising_s* g = b->inst[i];
            cap = std::min(cap, n > 0 ? words_cap(g, n) : 1LL);
            gr.smem_plain = std::max(gr.smem_plain, g->fast_smem);
            gr.smem_fused = std::max(gr.smem_fused, g->smem_fused);
            gr.max_S = std::max(gr.max_S, g->S);
            gr.max_R = std::max(gr.max_R, g->R);
        }
        for (int i : gr.ids) {
            int32_t rc = ensure_buffers(b->inst[i], cap, cap);
            if (rc)
                return rc;
        }
        const std::vector<Op> ops = plan(b->inst[gr.ids[0]], n, swap_every, cap);
        if (gr.key.kind == 2) {  // generic kernel: per-instance launches at capture time
            for (const Op& op : ops)
                gr.ops.push_back({op});
            continue;
        }
        for (const Op& op : ops) {
            BatchOp bo{op};
            std::vector<BatchItem> items;
            int32_t rc = ISING_OK;
            if (op.kind == Op::GEN) {
                std::vector<MtGenArgs> args;
                for (int j = 0; j < int(gr.ids.size()); ++j) {
                    int blocks = 0;
                    const MtGenArgs a = gen_args(b->inst[gr.ids[j]], op, &blocks);
                    args.push_back(a);
                    for (int k = 0; k < blocks; ++k)
                        items.push_back({j, a.first_stream + k});
                }
                const MtGenArgs* d = nullptr;
                rc = upload_raw(run->bufs, args, &d);
                bo.args = d;
            } else if (op.kind == Op::PT) {
                std::vector<PtArgs> args;
                for (int i : gr.ids)
                    args.push_back(pt_args(b->inst[i], op));
                const PtArgs* d = nullptr;
                rc = upload_raw(run->bufs, args, &d);
                bo.args = d;
                bo.n_items = int(args.size());
            } else {
                std::vector<SweepArgs> args;
                for (int j = 0; j < int(gr.ids.size()); ++j) {
                    ising_s* g = b->inst[gr.ids[j]];
                    args.push_back(sweep_args(g, op));
                    for (int k = 0; k < g->blocks; ++k)
                        items.push_back({j, k});
                }
                const SweepArgs* d = nullptr;
                rc = upload_raw(run->bufs, args, &d);
                bo.args = d;
            }
            if (!rc && !items.empty()) {
                bo.n_items = int(items.size());
                rc = upload_raw(run->bufs, items, &bo.items);
            }
            if (rc)
                return rc;
            gr.ops.push_back(bo);
        }
    }

    // ---- record: fork to the side streams, one group per branch, join
    if (!b->cap) {
        CK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
        b->side.resize(kBatchSide);
        b->join.resize(kBatchSide);
        for (int k = 0; k < kBatchSide; ++k) {
            CK(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming));
        }
    }
    const int nside = std::min<int>(kBatchSide, std::max<int>(1, int(order.size())));
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaEventRecord(b->fork, b->cap);
    for (int k = 0; k < nside && e == cudaSuccess; ++k)
        e = cudaStreamWaitEvent(b->side[k], b->fork, 0);
    int32_t rc = ISING_OK;
    for (int gi = 0; gi < int(order.size()) && e == cudaSuccess && !rc; ++gi) {
        BatchGroup& gr = *order[gi];
        cudaStream_t st = b->side[gi % nside];
        const GroupKey& k = gr.key;
        if (k.kind == 2) {
            std::vector<Op> ops;
            for (const BatchOp& bo : gr.ops)
                ops.push_back(bo.op);
            for (int i : gr.ids)
                if ((rc = enqueue(b->inst[i], ops, st)))
                    break;
            continue;
        }
        for (const BatchOp& bo : gr.ops) {
            if (bo.n_items == 0)
                continue;
            if (bo.op.kind == Op::GEN)
                e = launch_mt_gen_batch(static_cast<const MtGenArgs*>(bo.args), bo.items, bo.n_items,
                                        gr.max_S, st);
            else if (bo.op.kind == Op::PT)
                e = launch_pt_batch(static_cast<const PtArgs*>(bo.args), bo.n_items, gr.max_R, st);
            else
                e = launch_fast_batch(static_cast<const SweepArgs*>(bo.args), bo.items, bo.n_items,
                                      k.field_bits, k.rng, k.cmax, k.T,
                                      bo.op.kind == Op::FUSED ? gr.smem_fused : gr.smem_plain,
                                      k.lean, st);
            if (e != cudaSuccess)
                break;
        }
    }
    for (int k = 0; k < nside && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->join[k], b->side[k]);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(b->cap, b->join[k], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
    if (rc || e != cudaSuccess || e2 != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        if (rc)
            return rc;
        return cuda_fail(e != cudaSuccess ? e : e2, "recording the batch graph");
    }
    e = cudaGraphInstantiate(&run->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGraphInstantiate (batch)");
    return ISING_OK;
}

}  // namespace

extern "C" {

int32_t ising_batch_create(int32_t n_inst, const ising_instance_t* in, int32_t rng_mode,
                           int32_t field_bits, uint32_t flags, ising_batch_t* out)
{
    if (!out || !in || n_inst < 1)
        return fail(ISING_ERR_INVALID_ARG, "need n_inst >= 1 instances and an output pointer");
    *out = nullptr;
    if (flags & ~uint32_t(ISING_BATCH_PER_SWEEP))
        return fail(ISING_ERR_INVALID_ARG, "unknown batch flags");
    ising_batch_s* b = new ising_batch_s();
    long long words_per_sweep = 0;
    for (int i = 0; i < n_inst; ++i) {
        ising_t g = nullptr;
        int32_t rc = ising_create(in[i].n, in[i].row_ptr, in[i].col, in[i].J, in[i].h, in[i].n_slices,
                                  0u, &g);
        if (!rc) {
            g->packed_off = true;  // the packed kernel has no batched instantiation
            rc = replicas_init_impl(g, in[i].replicas, in[i].betas, in[i].seed, rng_mode, field_bits,
                                    uint32_t(i));
        }
        if (rc) {
            const std::string msg = "instance " + std::to_string(i) + ": " + g_err;
            if (g)
                ising_destroy(g);
            ising_batch_destroy(b);
            return fail(rc, msg);
        }
        b->inst.push_back(g);
        words_per_sweep += (long long)g->R * g->S * g->Mp * 4;
    }
    // pre-generated MT19937 words: about 8 GB for the whole batch, the same
    // number of sweeps per chunk for every instance
    const long long chunk = std::max<long long>(1, (8LL << 30) / std::max<long long>(words_per_sweep, 1));
    for (ising_s* g : b->inst)
        g->word_budget = chunk * (long long)g->R * g->S * g->Mp * 4;
    b->resident.resize(n_inst);
    for (int i = 0; i < n_inst; ++i)
        b->resident[i] = configure_instance(b->inst[i], true, 0) ? 1 : 0;
    b->packed = !(flags & ISING_BATCH_PER_SWEEP) && packed_batch_setup(b);
    *out = b;
    return ISING_OK;
}

int32_t ising_batch_set_stream(ising_batch_t b, void* s)
{
    if (!b)
        return fail(ISING_ERR_INVALID_ARG, "NULL batch");
    b->drop_runs();
    b->stream = static_cast<cudaStream_t>(s);
    for (ising_s* g : b->inst)
        ising_set_stream(g, s);
    return ISING_OK;
}

int32_t ising_batch_run(ising_batch_t b, int64_t n, int32_t swap_every)
{
    if (!b)
        return fail(ISING_ERR_INVALID_ARG, "NULL batch");
    if (n < 0)
        return fail(ISING_ERR_INVALID_ARG, "n must be >= 0");
    if (n == 0)
        return ISING_OK;
    const auto key = std::make_pair((long long)n, swap_every > 0 ? int(swap_every) : 0);
    auto it = b->runs.find(key);
    if (b->packed) {
        if (it == b->runs.end()) {
            ising_batch_s::Run run;
            const int32_t rc = packed_batch_build(b, n, key.second, &run);
            if (rc) {
                for (void* p : run.bufs)
                    cudaFree(p);
                return rc;
            }
            it = b->runs.emplace(key, run).first;
        }
        return packed_batch_launch(b, it->second);
    }
    if (it == b->runs.end()) {
        ising_batch_s::Run run;
        const int32_t rc = batch_record(b, n, key.second, &run);
        if (rc) {
            for (void* p : run.bufs)
                cudaFree(p);
            return rc;
        }
        it = b->runs.emplace(key, run).first;
    }
    CK(cudaGraphLaunch(it->second.exec, b->stream));
    return ISING_OK;
}

int32_t ising_batch_read_state(ising_batch_t b, int32_t inst, int8_t* spins, int32_t* fields,
                               int64_t* energy, int32_t* temp_of_slot, uint64_t* counters)
{
    if (!b || inst < 0 || inst >= int(b->inst.size()))
        return fail(ISING_ERR_INVALID_ARG, "no such instance");
    CK(cudaStreamSynchronize(b->stream));
    return ising_read_state(b->inst[inst], spins, fields, energy, temp_of_slot, counters);
}

int32_t ising_batch_read_swap_stats(ising_batch_t b, int32_t inst, uint64_t* accepted)
{
    if (!b || inst < 0 || inst >= int(b->inst.size()))
        return fail(ISING_ERR_INVALID_ARG, "no such instance");
    CK(cudaStreamSynchronize(b->stream));
    return ising_read_swap_stats(b->inst[inst], accepted);
}

int32_t ising_batch_get_info(ising_batch_t b, int32_t inst, ising_info_t* out, int32_t* resident)
{
    if (!b || inst < 0 || inst >= int(b->inst.size()))
        return fail(ISING_ERR_INVALID_ARG, "no such instance");
    if (resident)
        *resident = b->packed ? 1 : b->resident[inst];
    const int32_t rc = ising_get_info(b->inst[inst], out);
    if (rc || !b->packed || !out)
        return rc;
    for (const PackedWave& w : b->waves)  // the persistent packed launch of this instance
        if (std::find(w.ids.begin(), w.ids.end(), int(inst)) != w.ids.end()) {
            out->fast_kernel = 4;
            out->replicas_per_block = 1;
            out->threads_per_block = w.T;
            out->blocks = b->inst[inst]->R;
            out->smem_bytes = int(w.smem);
            out->persistent_ok = 1;
        }
    return ISING_OK;
}

int32_t ising_batch_destroy(ising_batch_t b)
{
    if (!b)
        return ISING_OK;
    b->drop_runs();
    dfree(b->d_bar);
    for (ising_s* g : b->inst)
        ising_destroy(g);
    for (cudaStream_t s : b->side)
        cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join)
        cudaEventDestroy(e);
    if (b->fork)
        cudaEventDestroy(b->fork);
    if (b->cap)
        cudaStreamDestroy(b->cap);
    delete b;
    return ISING_OK;
}

}  // extern "C"

namespace {

struct TuneCand {
    bool resident;
    int T, G;  // threads per block (0 = automatic), replicas per block when streamed
};

// SM-time of one sweep: measured time per sweep x blocks / blocks resident per
// SM (what the shape costs the GPU when many instances share it).
double tune_cost(ising_s* t, const TuneCand& c, bool* ok)
{
    *ok = false;
    const bool res = configure_instance(t, c.resident, c.T, c.G);
    if (c.resident != res || !t->use_fast)
        return 0.0;
    int per_sm = 0;
    if (fast_max_blocks_per_sm(t->field_bits, t->fast_cmax, t->rng, t->T,
                               res ? t->smem_fused : t->fast_smem, &per_sm, kernel_variant(t)) != cudaSuccess ||
        per_sm < 1)
        return 0.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return 0.0;
    double cost = 0.0;
    const int kSweeps = 4;
    if (ising_run(t, 2, 1) == ISING_OK && cudaEventRecord(e0, t->stream) == cudaSuccess &&
        ising_run(t, kSweeps, 1) == ISING_OK && cudaEventRecord(e1, t->stream) == cudaSuccess &&
        cudaEventSynchronize(e1) == cudaSuccess) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cost = double(ms) / kSweeps * double(t->blocks) / double(per_sm);
        *ok = true;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return cost;
}

}  // namespace

extern "C" int32_t ising_batch_autotune(ising_batch_t b, uint32_t flags)
{
    if (!b)
        return fail(ISING_ERR_INVALID_ARG, "NULL batch");
    if (flags != 0)
        return fail(ISING_ERR_INVALID_ARG, "flags must be 0");
    if (b->packed)
        return ISING_OK;  // persistent waves: the block shape follows from the slot counts
    std::map<std::tuple<int, int, int>, std::vector<int>> classes;
    for (int i = 0; i < int(b->inst.size()); ++i) {
        ising_s* g = b->inst[i];
        classes[std::make_tuple(g->S, g->M, pow2_at_least(g->R))].push_back(i);
    }
    for (auto& kv : classes) {
        ising_s* src = b->inst[kv.second[0]];
        ising_t t = nullptr;
        int32_t rc = ising_create(src->n, src->row_ptr.data(), src->col.data(), src->J.data(),
                                  src->h.data(), src->M, 0u, &t);
        if (!rc) {
            t->packed_off = true;  // the shapes of the batch's own instances (no packed kernel)
            rc = replicas_init_impl(t, src->R, src->betas.data(), src->seed, src->rng, src->field_bits,
                                    src->inst);
        }
        if (rc) {
            if (t)
                ising_destroy(t);
            return rc;
        }
        t->word_budget = src->word_budget;
        std::vector<TuneCand> cands = {{true, 0, 0}, {false, 0, 0}, {false, 0, 2}};
        // thread-count variants around the automatic choices
        for (bool res : {true, false}) {
            if (configure_instance(t, res, 0) != res)
                continue;
            const int T0 = t->T, step = std::max(32, t->G);
            for (int T : {T0 / 2, T0 * 2})
                if (T >= step && T <= 1024 && T % step == 0)
                    cands.push_back({res, T, 0});
        }
        double best = 0.0;
        TuneCand win{false, 0, 0};
        bool have = false;
        for (const TuneCand& c : cands) {
            bool ok = false;
            const double cost = tune_cost(t, c, &ok);
            if (ok && (!have || cost < best)) {
                best = cost;
                win = c;
                have = true;
            }
        }
        ising_destroy(t);
        cudaGetLastError();  // candidates that could not launch leave no sticky state
        if (!have)
            continue;
        for (int i : kv.second)
            b->resident[i] = configure_instance(b->inst[i], win.resident, win.T, win.G) ? 1 : 0;
    }
    b->drop_runs();
    return ISING_OK;
}

extern "C" int32_t ising_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda,
                                 const void* B, int32_t ldb, const float* bias, const void* mask,
                                 int32_t ldm, int32_t relu, void* C, int32_t ldc, int32_t c_bf16,
                                 void* stream)
{
    cudaError_t ce = device_setup();
    if (ce != cudaSuccess)
        return cuda_fail(ce, "device setup");
    static int* d_err = nullptr;
    if (!d_err && dalloc(&d_err, 1))
        return ISING_ERR_OOM;
    TcGemmArgs g{A, B, lda, ldb, M, N, K, bias, mask, ldm, relu, C, ldc, c_bf16, d_err};
    const cudaError_t e = launch_tc_gemm(g, static_cast<cudaStream_t>(stream));
    if (e == cudaErrorInvalidValue)
        return fail(ISING_ERR_INVALID_ARG,
                    "tc_gemm: M % 128, K % 64, N in {32,64,128,256}, leading dimensions % 8");
    if (e != cudaSuccess)
        return cuda_fail(e, "tc_gemm launch");
    return ISING_OK;
}
