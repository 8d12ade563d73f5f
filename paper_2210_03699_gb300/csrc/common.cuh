// Internal declarations of the GB300 CTR-IBIM engine (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "ctr_ibim.h"

namespace ctr {

// ---------------------------------------------------------------- constants
constexpr double kPi = 3.14159265358979323846;
constexpr int kModes = 9;          // Fourier modes k = 0, 2, ..., 16 (even: every l is even)
constexpr int kModeMax = 16;
constexpr int kSamples = 64;       // samples of l(theta) for the DFT, 4 * 16
constexpr int kTabHalf = 19;       // table shifts (i - 19)/32, i = 0..38
constexpr int kTabN = 2 * kTabHalf + 1;
constexpr double kTabSpacing = 1.0 / 32.0;
constexpr int kTabSize = 2 * kModes * kTabN * kTabN;

// device-side error word bits
enum : int { kErrWait = 1, kErrMargin = 2, kErrNumeric = 4, kErrCapacity = 8 };

// ---------------------------------------------------------------- errors
struct Error {
    int status;
    std::string msg;
};

void set_last_error(const std::string& msg);
int fail(int status, const std::string& msg);

#define CTR_CUDA_TRY(expr)                                                                  \
    do {                                                                                    \
        cudaError_t e_ = (expr);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            return ::ctr::fail(e_ == cudaErrorMemoryAllocation ? CTR_ERR_NOMEM : CTR_ERR_CUDA, \
                               std::string(#expr) + ": " + cudaGetErrorString(e_));         \
        }                                                                                   \
    } while (0)

// After every kernel launch: count it and surface launch errors.
void count_launch();
void count_launches(int64_t n);
#define CTR_LAUNCHED()                      \
    do {                                    \
        ::ctr::count_launch();              \
        CTR_CUDA_TRY(cudaGetLastError());   \
    } while (0)

#define CTR_TRY(expr)              \
    do {                           \
        int s_ = (expr);           \
        if (s_ < 0) return s_;     \
    } while (0)

// ---------------------------------------------------------------- device buffers
// Plain owning device allocation (cudaMalloc / cudaFree).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    int alloc(size_t n) {
        if (n <= bytes && p) return CTR_OK;
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return fail(CTR_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        bytes = n;
        return CTR_OK;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
};

// ---------------------------------------------------------------- node data
// Structure-of-arrays of the tube nodes in FP64 (one allocation).
struct NodeArrays {
    double *Px, *Py, *Pz, *nx, *ny, *nz, *W, *d;
    double *t1x, *t1y, *t1z, *t2x, *t2y, *t2z;  // principal directions
    double *m1, *m2;                           // M = diag(m1, m2) of the expansions
    static constexpr int kCount = 16;
};

// Pair-kernel launch plan of the one-sided grid launch (fixed-scratch entry point).
struct PairPlan {
    int R = 2;          // targets per thread
    int splits = 1;     // source splits (blockIdx.y)
    int src_per_split = 0;
    int target_blocks = 0;
};

// A work item of a pair schedule: target block I (BS consecutive nodes) against
// sources [j_begin, j_end); one-sided (sym = 0: correction pairs masked) or
// symmetric (sym = 1: both orientations of every pair, no correction pair in
// the item).  Its target sums (and a symmetric item's source sums) are added
// into the handle's exact per-node accumulators.
struct PairItem {
    int32_t I, j_begin, j_end, sym;
};

// The pair schedule of one system for one pair arithmetic: items (device list
// sorted by decreasing cost; host copy and costs kept for the engine).
struct PairSchedule {
    bool planned = false; // items built (an arithmetic the handle's options do not use is planned on first use)
    int var = 0;          // kernel variant (FP32: index into pk::kVar32; 0 for the fixed shapes)
    int R = 1;            // targets per thread
    int BS = 256;         // nodes per target block
    int tile = 128;       // sources per shared-memory tile
    int nb = 0;           // target blocks
    int64_t pairs_sym = 0, pairs_one = 0;   // evaluated pair orientations of each kind
    double total_cost = 0.0;                // sum of the item costs
    std::vector<PairItem> items;   // in the order of d_items (decreasing cost)
    std::vector<double> cost;
    DevBuf d_items;
};

// Throughput of each pair arithmetic ([0] FP32, [1] float-float, [2] FP64) on the whole GPU in the cost
// units of a schedule (one-sided pair evaluations; a symmetric evaluation counts its relative cost),
// as measured on a GB300 at M = 178,575 (1.23e12, 1.25e11 and 1.55e10 pair interactions/s).  Used only
// to size work (item lengths, engine parts), never in the arithmetic.
constexpr double kUnitRate[3] = {7.9e11, 7.5e10, 9.0e9};
// Longest item per arithmetic: this many seconds of one resident block at the rates above.  Short
// items keep the tail of a persistent launch short and let the engine split a large system's
// application into parts (an FP32 application of 180k nodes takes 26 ms, a float-float one 256 ms).
constexpr double kItemSeconds[3] = {8e-3, 4e-3, 4e-3};

// ---------------------------------------------------------------- far field (treecode)
constexpr int kTreeMaxN1 = 13;                                        // degree <= 12
constexpr int kTreeMaxNp = kTreeMaxN1 * kTreeMaxN1 * kTreeMaxN1;

// Far item: target block I against the far clusters flist[l0 .. l1); its sums are
// added into the nodes' exact accumulators (like a one-sided pair item's).
struct FarItem {
    int32_t I, l0, l1, pad;
};
// Moment chunk: the tree positions [j0, j1) of far cluster q (compact index).
struct MomChunk {
    int32_t q, j0, j1, pad;
};

// Device view of a handle's far-field data, per pair arithmetic p (0 FP32,
// 1 float-float, 2 FP64; moments and charges are FP32 for p = 0 and FP64 for p = 1, 2, far sums
// FP32, float-float and FP64; each arithmetic has its own interpolation degree n = n1 - 1).
struct TreeView {
    int on = 0;
    int M = 0;
    int n1[3] = {}, np[3] = {};           // points per axis, proxies per cluster
    const int32_t* tinv = nullptr;        // node -> tree position
    const double* xref[3] = {};           // n1 Chebyshev points cos(m pi / n)
    const double* bw[3] = {};             // n1 barycentric weights
    const double* dref[3] = {};           // n1 x n1 differentiation matrix, D[m * n1 + q] = l_q'(x_m)
    const double* box[3] = {};            // per far cluster: centre[3], half-width[3]
    const MomChunk* chunks[3] = {};
    const int32_t* cptr[3] = {};          // chunks of far cluster q: [cptr[q], cptr[q+1])
    void* mpart[3] = {};                  // per chunk: D[np], S[np]
    void* mom[3] = {};                    // per far cluster: Q0[np], Qk[np], Qk'[np]
    const FarItem* far[3] = {};
    const int32_t* flist[3] = {};         // far cluster (compact index) lists
    const float2* exp_tab = nullptr;      // float-float e^{-x} tables of the device (float-float far field)
    const float4* src32 = nullptr;        // the handle's packed sources, tree order
    const float4* srcdf = nullptr;
    const double4* src64 = nullptr;
    unsigned long long* acc = nullptr;    // exact node accumulators (shared with the pair items)
    int BS[3] = {};
    double c1 = 1.0, c2 = 1.0, kappa = 0.0;
};

// Host side of a handle's treecode (owns the device buffers the view points to).
struct TreeData {
    int leaf = 128, g = 2;
    int64_t n_clusters = 0;
    std::vector<int32_t> perm;            // node at each tree position
    DevBuf d_tinv, d_eptr, d_excl;        // node -> position; exclusion CSR in tree positions
    DevBuf d_counters, d_view;
    struct Pol {
        int degree = 10, n1 = 11, np = 1331;
        double theta = 0.8;
        DevBuf d_xref, d_bw, d_dref;
        int nq = 0;                                      // far clusters with charges
        int64_t near_pairs = 0, far_evals = 0, far_pairs = 0;
        std::vector<FarItem> far;                        // device order (decreasing cost)
        std::vector<double> far_cost;
        std::vector<MomChunk> chunks;                    // device order (decreasing cost)
        std::vector<double> chunk_cost;
        DevBuf d_box, d_chunks, d_cptr, d_mpart, d_mom, d_far, d_flist;
        DevBuf d_ent_mom, d_ent_red, d_ent_far;          // single-system work entries {0, index}
    } pol[3];
    TreeView view;                        // host copy of d_view
};

// Per-handle GMRES workspace.
struct Krylov {
    int m = 0;           // restart length
    int64_t n = 0;       // vector length 2M
    DevBuf V;            // (m+1) x n
    DevBuf H;            // (m+1) x m, column-major by column j: H[j*(m+1) + i]
    DevBuf cs, sn, s;    // Givens and rhs of the least-squares problem
    DevBuf y;            // m
    DevBuf part;         // partial dot products: (m+1) x nblk
    DevBuf scal;         // scalars: [0] beta, [1] hnorm, [2] residual estimate, [3] converged flag ...
    int nblk = 0;
};

}  // namespace ctr

// The handle behind the opaque C type.
struct ctr_ibim {
    int device = 0;
    cudaStream_t stream = nullptr;
    ctr_options opt{};
    int64_t n[3]{};
    double origin[3]{};
    double h = 0, eps = 0, eps_in = 1, eps_out = 1, kappa = 0;
    int64_t M = 0, E = 0;
    int64_t nc = 0;

    ctr::DevBuf lin;         // int64 [M] grid index
    ctr::DevBuf nodes;       // double [16][M]
    ctr::NodeArrays na{};
    ctr::DevBuf src32;       // float4 [4M]: {x,x,y,y} {z,z,a,a} {nx,nx,ny,ny} {nz,nz,-b,-b} (f32x2 operands)
    ctr::DevBuf src64;       // double4 [2M]
    ctr::DevBuf srcdf;       // float4 [4M]: float-float {P.hi, a.hi} {P.lo, a.lo} {n.hi, b.hi} {n.lo, b.lo}
    ctr::DevBuf corr_ptr;    // int32 [M+1]
    ctr::DevBuf corr_node;   // int32 [E]
    ctr::DevBuf corr_w;      // double [4][E]: omega11, omega21, omega22, omega12
    ctr::DevBuf bad;         // uint8 [M] hybrid classification
    ctr::DevBuf excl;        // int32 [E] sorted correction nodes per target
    ctr::DevBuf rhs;         // double [2M]
    ctr::DevBuf charges;     // double [4][nc]: x, y, z, q
    ctr::DevBuf acc;         // exact accumulators of the dense sum: pk::kFxWords x M 64-bit words
    ctr::DevBuf map_ws;      // double split partials of the potential-map kernels (grown on demand)
    ctr::DevBuf map_io;      // device staging of host arguments of the potential maps (grown on demand)
    ctr::DevBuf err;         // int device error word
    ctr::DevBuf vecs;        // double [6][2M] solver vectors
    ctr::DevBuf red;         // reduction scratch
    ctr::PairSchedule sched[3];   // pair schedules: [0] FP32, [1] float-float, [2] FP64
    ctr::DevBuf counter;          // int [4] work counters of the single-system launches
    ctr::Krylov kr;
    std::unique_ptr<ctr::TreeData> tree;   // far-field acceleration (farfield = CTR_FARFIELD_TREECODE)
};

namespace ctr {

// setup.cu
int setup_tube_and_geometry(ctr_ibim* s, const double* d_sdist);
int setup_rhs(ctr_ibim* s);
// weights.cu
int weight_tables_device(double* d_tables, cudaStream_t st);
int weight_tables_cached(int device, cudaStream_t st, const double** out);
int setup_corrections(ctr_ibim* s, const double* d_tables, const int32_t* d_node_of);
// pairsum.cu
int plan_pairs(ctr_ibim* s);
// tree.cu: the treecode of a handle (tree order, schedules, far-field data) and its
// single-system far-field launches for pair arithmetic pol
int build_tree_schedules(ctr_ibim* s, const int slots[3]);
int launch_tree(ctr_ibim* s, int pol);
int64_t tree_bytes(const ctr_ibim* s);
// schedule.cu: symmetric / one-sided pair schedules of a handle
int build_schedules(ctr_ibim* s, const int slots[3]);
int ensure_schedule(ctr_ibim* s, int pol);   // plans pair arithmetic `pol` if it has not been planned yet
// the handle's exact node accumulators, allocated and cleared (pairsum.cu)
int alloc_accumulators(ctr_ibim* s);
// the weights a = h^3 W x1 / (4 pi), b = h^3 W x2 / (4 pi) of x (2M doubles, device) into the packed
// sources of one arithmetic (pairsum.cu)
int pack_sources(ctr_ibim* s, const double* d_x, int precision);
int apply_operator(ctr_ibim* s, const double* d_x, double* d_y, int precision);
int apply_operator_timed(ctr_ibim* s, const double* d_x, double* d_y, int precision, cudaEvent_t* ev);
// krylov.cu: solver workspace
// potential.cu: psi_rxn of Eq. (2.31) at n points in pair arithmetic `precision` (CTR_FP32_REFINE,
// CTR_DF64 or CTR_FP64), all pointers device memory; enqueued on the handle's stream
int potential_map(ctr_ibim* s, const double* d_psi, const double* d_dpsi, int64_t n, const double* d_xyz,
                  double* d_out, int precision);
// reductions (krylov.cu)
int device_dot(ctr_ibim* s, const double* a, const double* b, int64_t n, double* h_out);
int check_device_error(ctr_ibim* s, const char* where);

// Exclusive scan of n int32 counts into offsets (n+1 entries, last = total), on stream.
int exclusive_scan_i32(const int32_t* d_counts, int32_t* d_offsets, int64_t n, cudaStream_t st,
                       DevBuf& scratch);

inline unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace ctr
