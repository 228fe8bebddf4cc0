// mps_internal.cuh -- shared declarations of the GB300 MPS library's translation units.
//
// Layout in HBM (all per-particle arrays are in the current Morton-sorted order, "slot" s):
//   pos, vel        double4 (x, y, z, 0)           FP64 master state
//   pos32           float4 (x-xmin, y-ymin, z-zmin, kind bits)   FP32 copy for filtering
//   type            int8, id int32 (caller's particle id of slot s)
//   pos_star/vel_star double4, pos32_star float4   predicted r*, u* of the step
//   pff_star        float4[2n]: r* as float-float, slot i's hi at 2 i and lo at 2 i + 1 (one
//                   32-byte sector per particle for the build's gathers)
//   pos32lo         float4 low parts: x - xmin = pos32.x + pos32lo.x to ~48 bits (float-float)
//   vl              sell8 rows of `cap_v` int32 slots: candidates within h at r^k (superset)
//   vel32           float4 velocities (mixed-precision viscosity terms)
//   nb_lap          sell8 rows of `cap` int32 slots: non-dummy neighbours within re_lap at
//                   r*, with the PPE coefficients c_ij: binary64 (v64, FP64 mode) or
//                   float-float hi/lo (v32/vlo, mixed mode; v32 is the FP32 coefficient)
//   nb_n            sell8 rows of `cap_n` int32 slots: non-dummy neighbours within re_n at r*
//   sell8: the rows of 32 consecutive slots form a slice, and a row's entries come in groups
//   of 8 (one 32-byte sector): entry k of row i sits at ((i / 32) cap + 8 (k / 8)) 32 +
//   8 (i % 32) + k % 8, so the 32 rows' group g is 1 KB contiguous, a row's run of
//   consecutive entries fills whole sectors, and a warp (one row per lane) reads a group of
//   its 32 rows with two 16-byte loads per lane.
//   cell_start      int32[2^(dim*bits) + 1], indexed by Morton code: exclusive scan of
//                   per-cell counts, so cell m holds slots [cell_start[m], cell_start[m+1])
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "mps.h"

namespace mps {

constexpr int kFluid = MPS_FLUID, kWall = MPS_WALL, kDummy = MPS_DUMMY, kGhost = MPS_GHOST;

// device error bits (DevStatus::err)
constexpr unsigned kErrCoincident = 1u, kErrCap = 2u, kErrNonfinite = 4u, kErrWait = 8u;
constexpr unsigned kErrKind = 16u;   // a particle kind outside FLUID..GHOST (state upload)

struct DevStatus {
    unsigned int err;
    unsigned int n_ghost;
    unsigned int n_occ;
    unsigned int n_surface;
    unsigned int n_ppe;
    unsigned int leave;                 // kept lists: particles whose next position leaves the grid or is not finite
    unsigned long long max_disp_bits;   // max squared FLUID displacement (bit pattern of a non-negative double)
    unsigned int counter[8];            // last-block-done tickets of grid reductions
    unsigned long long cand_tests;      // candidate distance tests of the cell gather
    unsigned long long pairs_lap;       // PPE coefficients evaluated (pairs within re_lap)
    unsigned long long pairs_n;         // number-density terms evaluated (pairs within re_n)
    unsigned long long max_disp_next_bits;   // kept lists: max squared |r^{k+1} - r_b| (as above)
    unsigned int gather_next;           // next occupied cell of the candidate gather (dynamic)
    unsigned int pad1;
    unsigned long long list_tests;      // candidate-list entries classified by the build (at r*)
    unsigned int n_fast;                // particles beyond half the full skin (skinpatch.cu)
    unsigned int differs;               // a written state differs from the context's
    unsigned int n_mov;                 // bucket build: particles whose cell key changed
    unsigned int pad2;
};

// Scalars of one CG solve; updated by the last block of each reduction kernel.
struct CgScalars {
    double rho;        // r.r of the current iterate
    double rho0;       // r.r at the (re)start of this solve
    double dq;         // d.q
    double alpha, beta;
    double rr;         // generic reduction result (residual norms)
    double stop2;      // stop when rho <= stop2
    int done;          // recurrence residual below the stop threshold
    int iters;         // iterations executed by this solve
    int max_iters;
    int pad;
    // device-driven mixed solve (one CUDA graph with conditional WHILE nodes): the outer
    // target, the refinement sweeps and inner iterations so far, their caps, the inner
    // tolerance, and loop guards that end either loop whatever the CG does
    double ostop2;
    double bb;         // |b|^2
    double inner_tol;
    int outer, total, max_outer, max_total;
    int guard_in, guard_out;
    double gw[4];      // initial guess x0 = sum_k gw[k] ph[k] (cg_x0 >= 1)
};

struct GridDesc {
    double bmin[3];
    double h;
    double inv_h;      // 1/h in binary64 (cell_floor)
    float inv_hf;      // 1/h rounded to binary32 (cell_floor's first tier)
    int ncell[3];
    int bits;
    int dim;
    uint32_t ghost_key;   // (number of scenes) << (dim*bits): sorts after every cell
};

// Precomputed bounds for the FP32 pre-filter of a distance predicate r^2 < re^2:
// r2_32 < lo  => certainly inside; r2_32 >= hi => certainly outside; else decide in FP64.
struct Radius {
    double re, re2;
    float lo, hi;       // FP32 band
    float re_f;
    float re2_h, re2_l; // re^2 as float-float
    float ff_tol;       // float-float band: |r2_ff - re^2| < ff_tol is decided in binary64
    float re_l;         // re = re_f + re_l (float-float)
    double inv_re;      // 1/re (the cubic weight (1 - r/re)^3)
    float inv_f, inv_l; // 1/re as float-float
};

// Per-scene constants of a batched ensemble (one entry per scene in device memory; a
// single-scene context has one).  The cell key of a particle is (scene << dim*bits) |
// Morton code of its cell in the shared grid, so each scene's particles are contiguous
// after the sort and the gathers never pair particles of different scenes.
struct SceneParams {
    Radius rn, rl, rv;          // predicates at re_n, re_lap and the candidate radius h_s
    double coef_lap, coef_ppe, coef_grad;
    double n0_pnd, n0_lap, lambda;
    float cre_h, cre_l;         // mixed build: coef_ppe re_lap and -coef_ppe as float-float
    float ncoef_h, ncoef_l;
    float cre2_h, cre2_l;       // the same with coef_lap (two-phase: the pair factor holds 1/rho)
    float ncoef2_h, ncoef2_l;
    double own_bmin[3];         // the scene's own grid (a particle outside it is a GHOST)
    double own_h;
    int own_ncell[3];
    int pad;
};

// Weight of kernel 1, (1 - r/re)^3 for r < re, from r^2 and 1/r (FP32 and binary64)
__device__ __forceinline__ float cubic_w_f(float r2, float rs, float inv_re) {
    const float t = fmaf(-(r2 * rs), inv_re, 1.f);
    return t * t * t;
}
__device__ __forceinline__ double cubic_w_d(double r2, double rs, double inv_re) {
    const double t = fma(-(r2 * rs), inv_re, 1.0);
    return t * t * t;
}

// The candidate lists and the PPE and gradient rows, in slices of 32 rows whose entries come
// in groups of 8 per row: entry k of row i at slice (i / 32), group (k / 8), row (i % 32),
// position (k % 8).  A row's group is one 32-byte sector (written whole by the build's
// thread, or as a run of consecutive entries by the gather's warp) and is read with two
// 16-byte loads; the 32 rows' group g is 1 KB contiguous.  cap is a multiple of 8.
__host__ __device__ __forceinline__ size_t sell8(int i, int k, int cap) {
    return ((size_t)(i >> 5) * (size_t)cap + (size_t)(k & ~7)) * 32 + (size_t)(i & 31) * 8 +
           (size_t)(k & 7);
}
// the first entry of row i (group g of the row sits 256 entries after group g - 1)
__host__ __device__ __forceinline__ size_t sell8_row(int i, int cap) { return sell8(i, 0, cap); }
__host__ __device__ __forceinline__ size_t sell_size(int64_t n, int cap) {
    return (size_t)((n + 31) / 32) * 32 * (size_t)cap;
}

struct Ctx;

// ---------------------------------------------------------------- bucket.cu
int bucket_build(Ctx* c, bool mutate);            // keys, sort, cell table, permute
void bucket_graphs_destroy(Ctx* c);
// end a stream capture left open by a failed capture (its result is discarded)
void abort_capture(Ctx* c);
void launch_cell_keys_only(Ctx* c, uint32_t* out_key);

// ---------------------------------------------------------------- scan.cu
// exclusive scan of m uint32 values; writes out[m] = total when write_total.
// Returns the number of kernels launched.
int scan_exclusive(const uint32_t* in, uint32_t* out, int64_t m, bool write_total,
                   uint32_t* scratch, cudaStream_t s);
int64_t scan_scratch_words(int64_t m);

// ---------------------------------------------------------------- gather.cu
void launch_copy_state_star(Ctx* c);
void launch_verlet(Ctx* c);
void launch_debug_neighbors(Ctx* c, const Radius& r, const int64_t* row_off, int32_t* out_ids,
                            int32_t* out_cnt);

// ---------------------------------------------------------------- rows.cu
void launch_predict_rows(Ctx* c);
void launch_build_rows(Ctx* c);
// zeros in the build's per-slot outputs (n*, flag, diagonal, right-hand side, list counts;
// p on the equation-of-state path): the slots it does not visit keep them
void launch_clear_rows(Ctx* c);
// threads per block of the row build; the functions' shared-memory limits (once per context)
int build_block_of(const Ctx* c);
int build_rows_init(Ctx* c);

// ---------------------------------------------------------------- ppe.cu
int ppe_solve(Ctx* c, mps_report* rep);
// the same solver on A x = b for another right-hand side (the adjoint solve); leaves the
// context's record of the step's PPE solve (iteration heuristic, residual) untouched
int ppe_solve_rhs(Ctx* c, double* x, const double* b, mps_report* rep);
void ppe_graphs_destroy(Ctx* c);
int ppe_time_kernel(Ctx* c, int which, int repeats, double* ms, double* bytes);

// ---------------------------------------------------------------- adjoint.cu
void launch_adj_mark(Ctx* c);
void launch_adj_load(Ctx* c, const double* d_gpos, const double* d_gvel);
void launch_adj_front(Ctx* c);
void launch_adj_back(Ctx* c, double* d_gsum);
void launch_adj_store(Ctx* c, double* d_out_r, double* d_out_u, double* d_out_nu);

// ---------------------------------------------------------------- update.cu
// the mixed solve's nodes appended to a graph (ppe.cu), its start scalars and kernel count
int add_mixed_solve(Ctx* c, cudaGraph_t G, cudaGraphNode_t dep, double* x, bool guess,
                    cudaGraphNode_t* last);
void mixed_init_scalars(Ctx* c, CgScalars* init);
int64_t mixed_solve_launches(Ctx* c, bool guess, const CgScalars& h);
// the stepping bucket build's launches and the state buffer assignment (bucket.cu)

constexpr size_t kPtrRecord = 24 * sizeof(void*);
void state_ptrs_save(const Ctx* c, void* rec);
void state_ptrs_load(Ctx* c, const void* rec);
// the candidate and predicate bands of radius re for coordinates up to X (api.cu)
Radius make_radius(double re, double X);
// candidate lists completed for particles beyond the full skin (skinpatch.cu)
int skin_patch_cap(const Ctx* c);
void launch_fast_mark(Ctx* c, double half);
int launch_fast_patch(Ctx* c, int n_fast, float hv2);
// whole steps as CUDA graphs (stepgraph.cu)
bool step_graph_eligible(const Ctx* c, bool advance);
// a conditional node of graph g after dep (null: none), its body graph in *body; the node a
// capture into stream s ends at (null unless exactly one)
int add_cond(Ctx* c, cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
             cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body);
cudaGraphNode_t capture_tail(cudaStream_t s);
// the bucket build appended to graph G after dep (bucket.cu); *tail: its last node
int bucket_append(Ctx* c, cudaGraph_t G, cudaGraphNode_t dep, cudaGraphNode_t* tail);
// kernels of the bucket build's branch that ran (after its status was read), into launches
void bucket_branch_count(Ctx* c, const DevStatus& st);
// the host's word for the next graph bucket build (before the graph's launch)
int bucket_order_word(Ctx* c);
int step_graph_step(Ctx* c, mps_report* rep);
int do_step(Ctx* c, bool advance, mps_report* rep);   // api.cu: the host-driven step
void step_graphs_destroy(Ctx* c);
void launch_clamp_pmin(Ctx* c);
// the clamp p = max(p, 0) of the PPE solution and p_hat of the gradient (update.cu)
int launch_pressure_floor(Ctx* c);
// the PPE solution before the clamp into the guess history (ph[0]), the older ones shifted
void launch_push_history(Ctx* c);
void launch_gradient_correct(Ctx* c);
void launch_unpermute(Ctx* c, double* d_pos, double* d_vel, double* d_p, double* d_nstar,
                      uint8_t* d_flags, int8_t* d_types);
void launch_ingest(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types,
                   bool keep_vel, bool keep_types);
// FP32 hi/lo split of a coordinate relative to the grid origin (float-float)
__device__ __forceinline__ void split_rel(double x, double xmin, float* hi, float* lo) {
    const double r = x - xmin;
    const float h = (float)r;
    *hi = h;
    *lo = (float)(r - (double)h);
}
void launch_unpermute_u32(Ctx* c, const uint32_t* in, uint32_t* out);
void launch_gather_props(Ctx* c);
void launch_ecs_rates(Ctx* c);
void launch_check_stage(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types);
void launch_same_state(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types);

// smallest skin of the candidate lists (relative to max(re)): the next gather takes three
// times what the last step's largest displacement needs, never less than this
constexpr double kMinListSkin = 0.02;

// ---------------------------------------------------------------- context
// The mixed PPE solve captured as one CUDA graph (outer refinement loop around the inner
// FP32 CG loop, both conditional WHILE nodes set by the kernels), one per buffer that the
// solution p can live in (the bucket build swaps p with its alternate buffer).
struct PpeGraph {
    const double* x = nullptr;
    const double* x0 = nullptr;   // the initial guess (cg_x0 = 1), or null: x0 = 0
    bool guess = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// The stepping bucket build captured as a CUDA graph, one per starting state buffer, with
// the buffer assignment it leaves behind (a record of pointers, see bucket.cu).
struct BucketGraph {
    const double4* pos = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;
    void* after[24] = {};
};

// Per-step control block of a step run as one CUDA graph (stepgraph.cu): written by the
// host into pinned memory and copied to the device before each launch (the host part), then
// updated by the graph's own kernels (the device part).
struct StepCtl {
    CgScalars cg_init;   // host: start values of the mixed solve's scalars
    double g[3];         // host: external acceleration of this step
    double half[2];      // host: s' max(re)/2 of the adaptive list skin s' (0) and of cell_skin (1)
    float hv2[2];        // host: single scene: the candidate bound of the two skins
    int can_retry;       // host: the adaptive skin is below cell_skin
    int attempt;         // device: 0, or 1 after a retry with the full skin
    int skin_err;        // device: a particle outran the full skin (MPS_ESKIN)
    float hv2_live;      // device: the bound the gather reads
};

// One step as a CUDA graph, one per starting state buffer (the bucket build alternates the
// buffers), with the buffer assignment it leaves behind and its kernel counts.
struct StepGraph {
    const double4* pos = nullptr;
    bool kept = false;   // a step on kept candidate lists: no bucket build, no gather
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_pre = 0, launches_attempt = 0, launches_post = 0;
    bool guess = false;
    void* after[24] = {};
};

// Work arrays of the reverse step (slot order unless noted), allocated on first use.
struct AdjBuffers {
    bool ready = false;
    double4 *gr = nullptr, *gu = nullptr;     // cotangents of r^{k+1}, u^{k+1}
    double4 *gG = nullptr;                    // of the pressure gradient (FLUID rows)
    double4 *grs = nullptr, *gus = nullptr;   // of r*, u*
    double4 *out_r = nullptr, *out_u = nullptr;
    double *gphat = nullptr, *pbar = nullptr, *lam = nullptr, *gn = nullptr;
    double* ppre = nullptr;                   // the PPE solution before the clamp
    int32_t* amin = nullptr;                  // slot giving p_hat of each FLUID row
    uint8_t* was_ghost = nullptr;             // by particle id: GHOST before the step
    double* gsum = nullptr;                   // dL/dg (3)
    double* gnu = nullptr;                    // dL/dnu of every slot (0 off FLUID)
};

struct Ctx {
    mps_params prm;
    int64_t n;
    int dim;
    int sms;
    cudaStream_t stream;
    bool own_stream;
    std::string last_error;
    std::vector<void*> allocations;

    // derived constants
    double n0_pnd, n0_lap, lambda, h;
    double coef_lap;     // 2d/(n0_lap lambda)            (Eq. 7)
    double coef_ppe;     // 2d/(n0_lap lambda rho)        (PPE coefficient)
    double coef_grad;    // d/n0_pnd                      (gradient)
    double diag_add;     // alpha_c/dt^2
    double inv_dt2;
    int cap, cap_n, cap_v;
    GridDesc grid;
    int64_t ntable;      // 2^(dim*bits)
    int sort_bits;
    Radius r_n, r_lap, r_v;   // r_v: candidate radius h (only r_v.hi is used)
    int64_t steps_done;
    int last_cg_iters;
    // candidate lists kept across steps (list_every > 1): positions r_b where they were
    // gathered, advanced steps since then, and whether the next step must gather afresh
    double4* pos_b = nullptr;
    int list_age = 0;
    bool need_list = true;
    int64_t n_ghost_last = 0;
    // reverse step: the forward it repeats gathers candidate lists for DUMMY rows too and
    // keeps the PPE solution before the clamp
    bool vjp = false;
    AdjBuffers adj;
    PpeGraph ppe_graph[2];
    BucketGraph bucket_graph[2];
    // whole steps as CUDA graphs (stepgraph.cu): the control block (device and pinned host
    // mirror), the two scene tables of an ensemble (adaptive and full list skin), the pinned
    // copy of the per-scene residual sums, and the control block kernels read while a step
    // is being captured (null otherwise)
    StepGraph step_graph[4];   // (starting buffer) x (fresh lists, kept lists)
    StepCtl* ctl = nullptr;
    StepCtl* ctl_host = nullptr;
    Radius* rv_var = nullptr;          // ensemble: candidate radius of every scene, 2 skins
    Radius* rv_var_host = nullptr;     // pinned staging of the adaptive half
    double* scene_sums_host = nullptr;
    double rv_var_skin = -1.0;         // the adaptive skin the device table holds
    StepCtl* capture_ctl = nullptr;
    // particles that outran the full skin in this step (skinpatch.cu), and whether the step
    // runs launch by launch (a step graph hands such a step to the host-driven path)
    int32_t* fast_idx = nullptr;
    bool force_host = false;
    // a graph capture failed (a launch refused inside it): every later step runs launch by
    // launch, and the graph of the failed capture is left alone (not destroyed: the runtime
    // may have dropped the body it was capturing into)
    bool graphs_off = false;

    // state (sorted order) and double buffers
    double4 *pos, *vel, *pos_alt, *vel_alt;
    int8_t *type, *type_alt;
    int32_t *id, *id_alt;
    double *p, *p_alt;
    // cg_x0 >= 1: the last guess_m solutions before the clamp (ph[0] the latest), of which
    // guess_n are valid (0 before the first solve and after a written state)
    static constexpr int kGuessMax = 4;
    double* ph[kGuessMax] = {};
    double* ph_alt[kGuessMax] = {};
    int guess_m = 0, guess_n = 0;
    float4 *pos32, *pos32lo;
    // step buffers
    double4 *pos_star, *vel_star;
    float4 *pos32_star, *pff_star;   // r* in FP32, and as (hi, lo) pairs (slot i at 2 i, 2 i + 1)
    float4* vel32;
    double* nstar;
    uint8_t* flag;
    double* bvec;
    double* diag;        // PPE diagonal; 0 on rows outside the PPE
    float* diag32;
    int32_t *vl_col, *vl_cnt;     // candidate (Verlet) lists at r^k, radius h
    int32_t *nb_lap_col, *nb_lap_cnt, *nb_n_col, *nb_n_cnt;
    double* nb_lap_v64;     // FP64 mode: binary64 coefficients
    float* nb_lap_v32;      // mixed mode: coefficient = v32 + vlo (float-float; v32 alone
    float* nb_lap_vlo;      //   is the FP32 coefficient of the inner solve)
    double* phat;
    // bucket build
    uint32_t *key, *key_alt;
    int32_t *perm, *perm_alt;
    uint32_t* hist;        // radix digit histograms
    uint32_t* hist_scan;
    uint32_t* cell_count;
    int32_t* cell_start;
    uint32_t* occ;         // occupied cell codes
    // bucket build from the previous order (bucket.cu): the slots whose key changed (flag
    // per slot, and up to mov_cap of them as (key, slot)), their counts and ranks, the
    // movers sorted by slot and by (key, slot); order_ok (device word, set by the host
    // before a build): the slot order is sorted by the keys and cell table in key/cell_start
    uint8_t* mvf = nullptr;
    uint32_t* mov_key = nullptr;
    int32_t* mov_slot = nullptr;
    uint32_t* mov_cnt = nullptr;       // 4 per mover
    int32_t* mov_by_slot = nullptr;
    unsigned long long* mov_by_key = nullptr;
    int32_t* order_ok = nullptr;
    int mov_cap = 0;
    bool order_valid = false;          // host: what order_ok is set to before the next build
    int64_t bucket_inc_launches = 0, bucket_radix_launches = 0;   // kernels of either branch
    int pending_branch = -1;   // a graph bucket build ran with this order_ok, branch not counted
    int last_bucket_merged = 0;   // the last bucket build merged its movers (1) or radix-sorted
    // two-phase flow: per-particle density / viscosity in original order (as given) and in
    // slot order (gathered by id after every reordering); null when uniform
    double *rho_id = nullptr, *nu_id = nullptr;
    double *rho_s = nullptr, *nu_s = nullptr;
    float2* rho_ff = nullptr;   // slot-order density as float-float (hi, lo)
    // active rows in slot order, rebuilt with every bucket build: FLUID slots (rows_f) and
    // FLUID or WALL slots (rows_fw); their counts sit after the exclusive scans
    uint32_t *mark_f, *mark_fw, *scan_f, *scan_fw;   // n + 1 each
    int32_t *rows_f, *rows_fw;
    double *ecs_nk = nullptr, *ecs_dk = nullptr;   // ECS source: n^k, (Dn/Dt)^k per row
    // batched ensemble: scenes, their constants (device table), the scene of every slot
    // (null for a single scene) and of every original particle, per-scene residuals
    int n_scenes = 1;
    std::vector<SceneParams> scn_host;
    SceneParams* scn = nullptr;
    uint16_t *sid = nullptr, *sid_id = nullptr;
    double* scene_sums = nullptr;        // 2 per scene: |r_s|^2, |b_s|^2
    std::vector<double> scene_resid;
    uint32_t scene_shift = 0;            // dim * bits
    double skin_half = 0.0;              // s max(re)/2 of the scene with the smallest spacing
    double re_skin = 0.0;                // max(re) of the scene with the smallest spacing
    double scn_skin = -1.0;              // ensemble: the list skin of the device scene table
    // Candidate-list skin of the next gather: sized from the last step's largest
    // displacement, at most cell_skin; X of the FP32 bands.
    double list_skin = 0.0;
    double gathered_skin = 0.0;          // the skin of the lists in use
    double band_x = 0.0;
    uint32_t* scan_scratch;
    // CG (FP64): x = p, r, d, q ; FP32: r32, d32, q32, x32
    double *cg_r, *cg_d, *cg_q;
    float *cg_r32, *cg_d32, *cg_q32, *cg_x32;
    float* cg_s32 = nullptr;   // the fused inner CG's A p (its A r is kept in cg_q32)
    // tuned by mps_autotune: the FP32 SpMV's block size and the inner CG's form
    int spmv_block = 512;
    bool cg_fused = false;
    int cg_unroll = 1;      // inner CG iterations per pass of the device-driven loop
    int build_block = 0;    // the row build's block (0: the path's default)
    int predict_tpr = 1;    // threads per row of the prediction (tuned: 1, 2 or 4)
    // capacities the grid-sized buffers were allocated with (the tuner's cell side may
    // derive smaller ones), and an ensemble's scenes (to derive its grid again)
    int cap_v_alloc = 0;
    int64_t ntable_alloc = 0;
    std::vector<mps_scene> scenes_host;
    float2* cg_xhl;         // mixed: the FP64 iterate as float-float (hi, lo) for the outer residual
    double* partials;       // per-block partial sums
    CgScalars* cg;          // device
    DevStatus* st;          // device
    DevStatus* st_host;     // pinned mirror
    CgScalars* cg_host;     // pinned mirror
    // staging for host transfers (original order)
    void* stage;
    size_t stage_bytes;
    // profiling: kernel launches issued, and per-stage CUDA-event timers
    int64_t launches;
    bool profiling;
    cudaEvent_t ev[2 * MPS_NSTAGES];
    double stage_ms[MPS_NSTAGES];
    int64_t stage_calls[MPS_NSTAGES];
};

// launch geometry
constexpr int kVecBlock = 256;
inline int vec_grid(const Ctx* c) { return c->sms * 4; }

// error helpers
int cuda_fail(Ctx* c, cudaError_t e, const char* what);
#define MPS_CUDA(c, call)                                        \
    do {                                                         \
        cudaError_t e__ = (call);                                \
        if (e__ != cudaSuccess) return ::mps::cuda_fail((c), e__, #call); \
    } while (0)

// ---------------------------------------------------------------- device helpers
__host__ __device__ inline uint32_t morton_encode(const int c[3], int dim, int bits) {
    uint32_t key = 0;
    for (int k = 0; k < bits; k++)
        for (int a = 0; a < dim; a++) key |= (uint32_t)((c[a] >> k) & 1) << (k * dim + a);
    return key;
}

__host__ __device__ inline void morton_decode(uint32_t key, int dim, int bits, int c[3]) {
    c[0] = c[1] = c[2] = 0;
    for (int k = 0; k < bits; k++)
        for (int a = 0; a < dim; a++) c[a] |= (int)((key >> (k * dim + a)) & 1u) << k;
}

// floor(fl(d / h)) -- the cell coordinate of the binary64 definition -- mostly without
// binary64 arithmetic, in three tiers:
//   1. binary32: qf = fl32(fl32(d) fl32(1/h)) carries three binary32 roundings, so
//      |qf - d/h| <= ~3 2^-24 |d/h| (1.8e-7 relative) and fl(d/h) is within 2^-53 of d/h:
//      both have the same floor unless qf lies within that of an integer (a margin of 2.7x:
//      4.8e-7 max(|qf|, 1)); qf - floor(qf) and floor(qf) + 1 - qf are exact;
//   2. binary64 q = fl(d fl(1/h)), within ~3 ulp of d/h: decided unless q lies within
//      4 ulp of an integer;
//   3. the (slow) binary64 division itself.
// Non-finite inputs fail both comparisons and reach the division.
__device__ __forceinline__ double cell_floor(double d, double h, double inv_h, float inv_hf) {
    const float qf = __fmul_rn(__double2float_rn(d), inv_hf);
    const float ff = floorf(qf);
    const float gapf = fminf(qf - ff, (ff + 1.0f) - qf);
    if (gapf > 4.8e-7f * fmaxf(fabsf(qf), 1.0f)) return (double)ff;
    const double q = d * inv_h;
    const double f = floor(q);
    const double gap = fmin(q - f, (f + 1.0) - q);
    if (gap > 4.0 * 2.220446049250313e-16 * fmax(fabs(q), 1.0)) return f;
    return floor(__ddiv_rn(d, h));
}

// Squared distance in binary64 with one rounding per operation and the fixed order
// ((dx*dx)+(dy*dy))+(dz*dz): no fused multiply-add, so the predicate r^2 < re^2 is
// decided identically to a plain IEEE evaluation of the definition.
__device__ __forceinline__ double exact_dist2(const double4& a, const double4& b) {
    double dx = __dsub_rn(b.x, a.x), dy = __dsub_rn(b.y, a.y), dz = __dsub_rn(b.z, a.z);
    double s = __dmul_rn(dx, dx);
    s = __dadd_rn(s, __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s;
}

// Classify a pair for radius r from its FP32 squared distance; only pairs inside the
// rounding band around re^2 are decided from the FP64 positions.
__device__ __forceinline__ bool in_radius(float r2, const Radius& r, const double4* pos, int i,
                                          int j, const double4& pi) {
    if (r2 < r.lo) return true;
    if (r2 >= r.hi) return false;
    return exact_dist2(pi, pos[j]) < r.re2;
}

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum (fixed tree); every thread must call it.  Returns the sum to
// all threads.
template <int BT>
__device__ __forceinline__ double block_sum(double v, double* smem /* >= BT/32 */) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = (lane < BT / 32) ? smem[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) smem[0] = t;
    }
    __syncthreads();
    t = smem[0];
    __syncthreads();
    return t;
}

// Grid reduction with a deterministic finish: each block stores its partial; the last
// block to arrive sums the partials in block order.  Returns true in the last block,
// where *total is valid (in every thread of that block).
template <int BT>
__device__ bool grid_sum(double block_partial, double* partials, unsigned int* counter,
                         double* total, double* smem) {
    __shared__ bool s_last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = block_partial;
        __threadfence();
        unsigned int t = atomicAdd(counter, 1u);
        s_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += BT) v += ((volatile double*)partials)[b];
    v = block_sum<BT>(v, smem);
    if (threadIdx.x == 0) *counter = 0u;
    *total = v;
    return true;
}

}  // namespace mps
