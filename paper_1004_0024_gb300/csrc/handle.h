// Internal state of a handle (host.cu); shared with the translation units
// that implement further entry points on handles (learned.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include <map>
#include <utility>
#include <vector>

#include "ising_gb300.h"

struct ising_s {
    double* d_betas = nullptr;       // [R] inverse temperatures by index
    float* d_betas32 = nullptr;      // [R] the same rounded to FP32
    unsigned long long learned_passes = 0;
    // colour classes of the slice graph for column moves (built on first use):
    // sites of class c are d_colour_sites[colour_off[c] .. colour_off[c+1])
    std::vector<int> colour_off, colour_sites;
    int* d_colour_sites = nullptr;
    int* d_sp_off = nullptr;  // [S+1] spatial neighbour list of each site
    int2* d_sp_nbr = nullptr; // (site, J) entries
    uint32_t* d_colbits = nullptr;  // [R][S] bit t = (spin (t, q) > 0), kept during a learned pass
    size_t colbits_cap = 0;         // entries of d_colbits (R * S of the replicas it was sized for)
    int sp_simd = 0;                // every site has sum_j 2 |J_qj| <= 127 over its spatial neighbours
    long long* d_obs = nullptr;  // [R] per-slot magnetisation (ising_read_observables)
    int* d_widen = nullptr;      // int32 scratch of ising_read_state (int16 fields), widen_cap entries
    size_t widen_cap = 0;
    // graph
    int n = 0, M = 1, S = 0, W = 1, Mp = 4, D0 = 0, D = 0, max_sp_deg = 0, max_sp_J = 0;
    long long kmax = 0, ebound = 0;
    std::vector<int> row_ptr, col, J, h;
    std::vector<int> site, pos, lev0p, jtau, nbr_off;
    std::vector<uint32_t> nbr;
    int *d_row_ptr = nullptr, *d_col = nullptr, *d_J = nullptr, *d_h = nullptr;
    int *d_nbr_off = nullptr, *d_jtau = nullptr, *d_lev0 = nullptr, *d_site = nullptr,
        *d_pos = nullptr;
    uint32_t* d_nbr = nullptr;
    // replicas
    bool inited = false;
    int R = 0, rng = 0, field_bits = 32, K = 1, maxpairs = 0;
    uint32_t seed = 0, inst = 0;
    std::vector<double> betas;
    bool pt_ok = true;  // false when the FP64 swap tables would exceed 2^28 entries
    int8_t* d_spins = nullptr;
    void* d_fields = nullptr;
    int *d_E = nullptr, *d_temp = nullptr, *d_slot = nullptr, *d_err = nullptr;
    unsigned long long *d_swap_acc = nullptr, *d_counters = nullptr, *d_mtpos = nullptr;
    unsigned* d_done = nullptr;
    uint32_t *d_thr = nullptr, *d_swthr = nullptr, *d_mtring = nullptr;
    long long* d_swoff = nullptr;
    int* d_swlen = nullptr;
    uint32_t *d_wbuf = nullptr, *d_swbuf = nullptr;
    int* d_Epub = nullptr;
    unsigned* d_gridbar = nullptr;
    // split couplings (ising_set_trotter; cleared by ising_replicas_init)
    bool split = false;
    int split_ks = 0;                  // k_space in [-split_ks, split_ks]
    std::vector<double> trotter_K;     // [R] by temperature index
    int* d_C = nullptr;                // [R] -sum over Trotter pairs of s s'
    int* d_Cpub = nullptr;             // [2][R]
    double *d_dbeta = nullptr, *d_dK = nullptr;  // [R-1]
    long long wbuf_cap = 0, swbuf_cap = 0;  // sweeps / passes
    long long word_budget = 8LL << 30;     // bytes of pre-generated MT19937 words
    // launch configuration
    int G = 1, T = 32, cmax = 1, blocks = 1, tables_smem = 1, thr_smem = 1, stage_words = 0;
    size_t smem = 0;
    // register-resident kernel (M <= 32, tables in shared memory)
    bool use_fast = false, use_lean = false, persistent_ok = false, fast_off = false, lean_off = false;
    bool use_track = false, track_on = false;
    int accept_mode = 0;      // ISING_ACCEPT_* of the flip thresholds (next replicas_init)
    bool lean_small = false;  // lean kernel, small-block instantiation (kernel variant 3)
    bool lean_long = false;   // lean kernel, long columns: M > 32 (kernel variant 4)
    // track schedule: columns (positions) in time order, track k =
    // track_col[track_off_v[k] .. track_off_v[k+1])
    std::vector<int> track_off_v, track_col;
    int ntracks = 0;
    int *d_track_off = nullptr, *d_track_col = nullptr;
    // packed kernel (packed_impl.cuh, kernel variant 5): columns packed into
    // slots whose busy windows do not overlap, slot k = slot_col[slot_off[k] ..
    // slot_off[k+1]); the device table buffer d_pk (pk_bytes) holds the column
    // descriptors, positions and slot lists
    std::vector<int> slot_off_v, slot_col_v;
    int nslots = 0;
    int sp_bound = 0;  // max over sites of |h_q| + sum of |J| over its spatial neighbours
    uint32_t* d_pk = nullptr;
    uint32_t pk_bytes = 0;
    bool use_packed = false, packed_off = false;
    int gen_slices = 4;  // the packed kernel's MT19937 staging: 4 slices, or 2 where 4 would not fit
    int fast_cmax = 1;
    size_t fast_smem = 0, smem_fused = 0;
    int G_req = 0, T_req = 0, allow_persistent = 1;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
    // statistics
    long long n_launches = 0, n_sweep_launches = 0;
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending;
    long long n_timed = 0;
    double kernel_ms = 0.0;
    std::map<std::pair<long long, int>, std::pair<long long, long long>> graph_counts;
    std::map<std::pair<long long, int>, cudaGraphExec_t> graphs;

    void free_replicas();
    void free_all();
    void drop_graphs();
};

int32_t isg_fail(int32_t code, const char* msg);
int32_t isg_device_setup();  // once per process: kernel attributes, SM count
int isg_num_sms();           // SMs of the current device (after isg_device_setup)
bool isg_pt_ok(const ising_s* g);
bool isg_alloc_allowed(size_t bytes);  // the cap of ising_set_alloc_cap
int32_t isg_noalloc_prepare();  // noalloc.cu: resolve the static scratch on the current device
