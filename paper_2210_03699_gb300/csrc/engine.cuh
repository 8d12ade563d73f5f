// Multi-slot solver engine (engine.cu): device-side state of every slot and the host object.
#pragma once

#include <memory>
#include <vector>

#include "common.cuh"
#include "pairkern.cuh"

namespace ctr {

// A slot whose operator application is split into parts (Engine::quantum_s) waits in kSlotInnerWait /
// kSlotUpdateWait between the steps that run its parts.
enum : int {
    kSlotEmpty = 0,
    kSlotInner = 1,
    kSlotUpdate = 2,
    kSlotDone = 3,
    kSlotStart = 4,
    kSlotInnerWait = 5,
    kSlotUpdateWait = 6
};

// Per-slot counters and state, read back by the host after every step.
struct SlotStat {
    int state;
    int converged;
    int numeric_error;
    int pad;
    int64_t iterations, refinements, matvecs_fp32, matvecs_fp64;
    double residual;
};

// Everything the step kernels need about one slot (device copy; the host mirror is Engine::host).
struct SlotDev {
    SlotStat stat;
    int j, m, kdone, cycle_end;
    int M, E, nblk;
    int64_t n;
    int refine, inner_prec, res_prec, max_refine;
    int res_update;          // refinement residuals after the first: r -= A d in the inner arithmetic
    int upd;                 // this cycle's residual is such an update (d = the cycle's correction, in z)
    int part;                // first part of the current operator application run in this step
    int span;                // parts run in this step (set by the step's planning kernel)
    int nparts[3];           // parts of one application per pair arithmetic (1: whole in one step)
    float part_s[3];         // estimated seconds of one part (of the whole application when nparts = 1)
    int64_t budget;
    // system (owned by the handle)
    const double* W;
    const int32_t* cptr;
    const int32_t* cnode;
    const double* cw;
    const int32_t* excl;     // excluded sources of each target, in the order of the packed sources
    const int32_t* eptr;     // ... and their row pointers (cptr, or the treecode's tree-order lists)
    const int32_t* tinv;     // treecode: node -> tree position of the packed sources (else NULL)
    float4* src32;
    double4* src64;
    float4* srcdf;
    unsigned long long* acc;   // exact node accumulators of the dense sum
    const double* g;
    double lam1, lam2, il1, il2, h2, h3, scale;
    pk::PairConsts kc;
    // pair schedules of the three arithmetics ([0] FP32, [1] float-float, [2] FP64; owned by the handle)
    const PairItem* items[3];
    int BS[3];
    TreeView tv;             // far-field data of a treecode handle (tv.on = 0 otherwise)
    // solver workspace (owned by the handle)
    double *x, *r, *z, *V, *H, *cs, *sn, *sv, *y, *cgs, *cgs2, *dpart, *scal;
    double gnorm, beta, tol_out, inner_tol, tol_cycle;
};

struct Engine {
    int device = 0;
    cudaStream_t stream = nullptr;
    int cap = 0;
    bool use_graph = true;
    bool graph_dirty = true;
    bool lists_dirty = false;   // slots admitted or retired since the work lists were built (engine_step rebuilds)
    int vec_blocks = 1;
    int max_nblk = 1;
    int max_m = 1;
    int sms = 1;
    // work lists per pair arithmetic and kernel variant (FP32: the variant of each slot's schedule)
    int64_t item_cap[3][pk::kNumVar32] = {};
    bool var_used[pk::kNumVar32] = {};   // FP32 variants of the occupied slots
    int64_t steps = 0;
    int64_t kernels_per_step = 0;
    // Part size (seconds at kUnitRate): an application expected to take longer is split into parts
    // (balanced sets of its schedule's items) run over consecutive steps, one or more per step (as
    // many as fit in the other slots' work of the step; k_plan_step), so that the steps of the other
    // slots do not wait for its whole application.  0: every application runs whole.  The exact node
    // accumulators make the result independent of the split.
    double quantum_s = 0.0;
    const float2* exp_tab = nullptr;
    bool kc_shared[3] = {false, false, false};   // all slots of an arithmetic share their pair constants
    pk::PairConsts kc_val[3] = {};               // ... and these are they (launch parameter)
    std::vector<SlotDev> host;
    std::vector<ctr_ibim*> owner;
    DevBuf slots, stats, items[3][pk::kNumVar32], n_items, counters, err;
    DevBuf need;   // per pair arithmetic: does any slot need its pair launch in the current half (k_need)
    // treecode work entries (slot, index) per pair arithmetic: moment chunks, far clusters, far items
    bool any_tree = false;
    int tree_np[3] = {0, 0, 0};   // largest proxy count per arithmetic among the treecode slots
    int64_t tree_cap[3][3] = {};
    DevBuf tree_ent[3][3], tree_cnt, tree_counters;
    cudaGraphExec_t graph_exec = nullptr;
    ~Engine();
};

int engine_create(int device, int cap, Engine** out);
int engine_admit(Engine* e, ctr_ibim* s, int* slot);
int engine_retire(Engine* e, int slot, ctr_solve_info* info);
int engine_step(Engine* e, std::vector<SlotStat>* stats);
int engine_prepare_handle(ctr_ibim* s);
int engine_solve_all(ctr_ibim* const* hs, int64_t n, int use_graph, std::vector<ctr_solve_info>* infos,
                     int64_t* steps);
int ensure_krylov_public(ctr_ibim* s);

}  // namespace ctr
