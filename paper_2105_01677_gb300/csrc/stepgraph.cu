// stepgraph.cu -- one time step as one CUDA graph: one launch and one stream
// synchronisation per step instead of ~70 launches and a status read in the middle.
//
//   status reset -> bucket build (Sec. 4.1), whose permutation also sets r* := r
//   WHILE (retry) {                                         at most two attempts
//       reset the attempt's counters, candidate radius of the attempt's skin
//       candidate lists -> prediction (Eq. 2, Eq. 7) -> n*, flags, PPE rows (Eq. 5, 15, 13)
//       check: an error, or a particle beyond the lists' skin -> retry once with the full
//       cell skin (as the host-driven step does), or MPS_ESKIN
//   }
//   IF (no error) {
//       PPE (Eq. 13): the device-driven mixed solve (its own nested WHILE nodes)
//       push the solution into the guess history, clamp + p_hat, gradient correction
//       (or, on the equation-of-state path, p_hat and the correction)
//   }
//   copies of the status word, the solver's scalars and the per-scene sums to pinned host
//
// The decisions the host-driven step takes between launches are taken by one-thread kernels
// that set the conditionals; everything the host changes from step to step (the adaptive
// list skin and its candidate radii, the acceleration, the guess weights) sits in a control
// block copied to the device before the launch, and the kernels that use it read it there
// while the graph is captured.  The kernels and their arithmetic are the host-driven step's,
// so both give identical results.  Used for single scenes and ensembles on the mixed path
// and the equation-of-state path, with candidate lists gathered every step and the stage
// timers off; the bucket build alternates the state buffers, so there is one graph per
// starting buffer.
#include <cmath>
#include <cstring>

#include "mps_internal.cuh"

namespace mps {

int add_cond(Ctx* c, cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
             cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    MPS_CUDA(c, cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &cp));
    *body = cp.conditional.phGraph_out[0];
    return MPS_OK;
}

// the node a capture into `s` currently ends at (null unless exactly one)
cudaGraphNode_t capture_tail(cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess)
        return nullptr;
    return nd == 1 ? deps[0] : nullptr;
}

namespace {

// the attempt's counters (the first attempt finds them zeroed by the step's status reset);
// the candidate bound or radii of the attempt's skin
// The loop's condition is cleared here and set again only by the check at the end of the
// attempt, so an attempt whose check does not run ends the loop.
__global__ void k_attempt_begin(StepCtl* ctl, DevStatus* st, SceneParams* scn, const Radius* var,
                                int n_scenes, cudaGraphConditionalHandle h_loop) {
    const int a = ctl->attempt;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        cudaGraphSetConditional(h_loop, 0u);
        ctl->hv2_live = ctl->hv2[a];
        st->n_surface = 0;
        st->n_ppe = 0;
        st->max_disp_bits = 0ull;
        st->cand_tests = 0ull;
        st->pairs_lap = 0ull;
        st->pairs_n = 0ull;
        st->list_tests = 0ull;
        st->gather_next = 0u;
    }
    if (var)
        for (int s = t; s < n_scenes; s += blockDim.x * gridDim.x) scn[s].rv = var[(size_t)a * n_scenes + s];
}

// after the build: errors end the step; a displacement beyond the lists' skin gathers again
// with the full skin once, and beyond the full skin ends the step with MPS_ESKIN
__global__ void k_attempt_check(StepCtl* ctl, const DevStatus* st, cudaGraphConditionalHandle h_loop,
                                cudaGraphConditionalHandle h_rest) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int a = ctl->attempt;
    const double disp = sqrt(__longlong_as_double((long long)st->max_disp_bits));
    bool loop = false, rest = false;
    if (st->err != 0u) {
        // reported from the status word
    } else if (disp > ctl->half[a]) {
        if (a == 0 && ctl->can_retry) {
            ctl->attempt = 1;
            loop = true;
        } else {
            ctl->skin_err = 1;
        }
    } else {
        rest = true;
    }
    cudaGraphSetConditional(h_loop, loop ? 1u : 0u);
    cudaGraphSetConditional(h_rest, rest ? 1u : 0u);
}

int alloc_ctl(Ctx* c) {
    if (c->ctl) return MPS_OK;
    StepCtl* d = nullptr;
    {
        void* p = nullptr;
        if (c->prm.alloc) {
            p = c->prm.alloc(std::max<size_t>(sizeof(StepCtl), 256), c->prm.alloc_user);
            if (!p) return MPS_ENOMEM;
        } else if (cudaMalloc(&p, sizeof(StepCtl)) != cudaSuccess) {
            cudaGetLastError();
            return MPS_ENOMEM;
        }
        c->allocations.push_back(p);
        d = (StepCtl*)p;
    }
    Radius* var = nullptr;
    const int S = c->n_scenes;
    if (S > 1) {
        void* p = nullptr;
        const size_t bytes = std::max<size_t>(2 * (size_t)S * sizeof(Radius), 256);
        if (c->prm.alloc) {
            p = c->prm.alloc(bytes, c->prm.alloc_user);
            if (!p) return MPS_ENOMEM;
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return MPS_ENOMEM;
        }
        c->allocations.push_back(p);
        var = (Radius*)p;
        if (cudaMallocHost(&c->rv_var_host, 2 * (size_t)S * sizeof(Radius)) != cudaSuccess ||
            cudaMallocHost(&c->scene_sums_host, 2 * (size_t)S * sizeof(double)) != cudaSuccess)
            return MPS_ENOMEM;
        // the full-skin half of the table does not change
        for (int s = 0; s < S; s++) {
            const SceneParams& sp = c->scn_host[(size_t)s];
            c->rv_var_host[(size_t)S + s] =
                make_radius(std::max(sp.rn.re, sp.rl.re) * (1.0 + c->prm.cell_skin), c->band_x);
        }
        MPS_CUDA(c, cudaMemcpyAsync(var + S, c->rv_var_host + S, sizeof(Radius) * (size_t)S,
                                    cudaMemcpyHostToDevice, c->stream));
        MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    if (cudaMallocHost(&c->ctl_host, sizeof(StepCtl)) != cudaSuccess) return MPS_ENOMEM;
    std::memset(c->ctl_host, 0, sizeof(StepCtl));
    c->ctl = d;
    c->rv_var = var;
    return MPS_OK;
}

// Capture the step for the current state buffers into graph G (build_step_graph restores
// the context's buffer assignment and counters whatever happens here).
int capture_step(Ctx* c, StepGraph* sg, cudaGraph_t G) {
    const mps_params& P = c->prm;
    const size_t n = (size_t)c->n;
    const bool ppe = P.pressure_mode == 0;
    cudaStream_t s = c->stream;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaGraph_t L = nullptr, R = nullptr, tmp = nullptr;
    cudaGraphConditionalHandle h_loop = 0, h_rest = 0;
    cudaGraphNode_t n_pre, n_loop, n_rest;
    int rc;
    // ---- status reset, the bucket build, r* := r
    int64_t l = c->launches;
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_loop, G, 1, cudaGraphCondAssignDefault));
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_rest, G, 0, cudaGraphCondAssignDefault));
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, nullptr, nullptr, 0, mode));
    MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), s));
    cudaGraphNode_t n_st = capture_tail(s);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    if (!n_st) return MPS_EDEVICE;
    if (sg->kept) {
        // kept candidate lists: the state stays in its order, r* := r copied
        MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, &n_st, nullptr, 1, mode));
        launch_copy_state_star(c);
        n_pre = capture_tail(s);
        MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
        if (!n_pre) return MPS_EDEVICE;
    } else {
        // (the bucket build's permutation also writes r* := r)
        if ((rc = bucket_append(c, G, n_st, &n_pre))) return rc;
        if (P.list_every > 1) {
            // the positions the lists are gathered at
            MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, &n_pre, nullptr, 1, mode));
            MPS_CUDA(c, cudaMemcpyAsync(c->pos_b, c->pos, n * sizeof(double4),
                                        cudaMemcpyDeviceToDevice, s));
            n_pre = capture_tail(s);
            MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
            if (!n_pre) return MPS_EDEVICE;
        }
    }
    sg->launches_pre = c->launches - l;
    // ---- WHILE (retry): candidate lists, prediction, build, check
    if ((rc = add_cond(c, G, n_pre, h_loop, cudaGraphCondTypeWhile, &n_loop, &L))) return rc;
    l = c->launches;
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, L, nullptr, nullptr, 0, mode));
    const int S = c->n_scenes;
    k_attempt_begin<<<S > 1 ? (S + 255) / 256 : 1, 256, 0, s>>>(c->ctl, c->st, c->scn,
                                                                 S > 1 ? c->rv_var : nullptr, S,
                                                                 h_loop);
    // the candidate-list counts of the slots the gather does not visit were zeroed by the
    // bucket build's permutation
    if (!sg->kept) launch_verlet(c);
    launch_predict_rows(c);
    if (ppe && P.source_term == 2) launch_ecs_rates(c);
    launch_clear_rows(c);
    launch_build_rows(c);
    k_attempt_check<<<1, 32, 0, s>>>(c->ctl, c->st, h_loop, h_rest);
    c->launches += 2;
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    sg->launches_attempt = c->launches - l;
    // ---- IF (no error): pressure and correction
    if ((rc = add_cond(c, G, n_loop, h_rest, cudaGraphCondTypeIf, &n_rest, &R))) return rc;
    l = c->launches;
    cudaGraphNode_t dep = nullptr;
    if (ppe) {
        MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, R, nullptr, nullptr, 0, mode));
        MPS_CUDA(c, cudaMemcpyAsync(c->cg, &c->ctl->cg_init, sizeof(CgScalars),
                                    cudaMemcpyDeviceToDevice, s));
        dep = capture_tail(s);
        MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
        if (!dep) return MPS_EDEVICE;
        sg->guess = c->guess_m > 0;
        if ((rc = add_mixed_solve(c, R, dep, c->p, sg->guess, &dep))) return rc;
    }
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, R, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                              mode));
    if (ppe && c->guess_m > 0) launch_push_history(c);   // the next solve starts from this one
    if ((rc = launch_pressure_floor(c))) return rc;
    launch_gradient_correct(c);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    sg->launches_post = c->launches - l;
    // ---- what the host reads after the step
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, &n_rest, nullptr, 1, mode));
    MPS_CUDA(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    MPS_CUDA(c, cudaMemcpyAsync(c->cg_host, c->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, s));
    MPS_CUDA(c, cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, s));
    if (ppe && S > 1)
        MPS_CUDA(c, cudaMemcpyAsync(c->scene_sums_host, c->scene_sums,
                                    2 * sizeof(double) * (size_t)S, cudaMemcpyDeviceToHost, s));
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    MPS_CUDA(c, cudaGetLastError());
    MPS_CUDA(c, cudaGraphInstantiate(&sg->exec, G, 0));
    return MPS_OK;
}

int build_step_graph(Ctx* c, StepGraph* sg) {
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned char before[kPtrRecord];
    state_ptrs_save(c, before);
    const int64_t l0 = c->launches;
    cudaGraph_t G = nullptr;
    MPS_CUDA(c, cudaGraphCreate(&G, 0));
    sg->graph = G;
    c->capture_ctl = c->ctl;
    int rc = capture_step(c, sg, G);
    c->capture_ctl = nullptr;
    if (rc) {
        abort_capture(c);
    } else {
        state_ptrs_save(c, sg->after);   // the assignment a replay leaves behind
    }
    state_ptrs_load(c, before);
    c->launches = l0;
    return rc;
}

}  // namespace

bool step_graph_eligible(const Ctx* c, bool advance) {
    const mps_params& P = c->prm;
    return P.step_graph == 1 && advance && !c->vjp && !c->profiling && !c->force_host &&
           !c->graphs_off &&
           (P.pressure_mode == 1 || (P.precision == 1 && P.ppe_host_loop == 0));
}

void step_graphs_destroy(Ctx* c) {
    for (StepGraph& g : c->step_graph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = StepGraph{};
    }
}

int step_graph_step(Ctx* c, mps_report* rep) {
    const mps_params& P = c->prm;
    const bool ppe = P.pressure_mode == 0;
    const double re_max = c->re_skin;
    int rc;
    if ((rc = alloc_ctl(c))) return rc;
    // candidate lists kept across steps (list_every > 1): a step on the kept lists runs the
    // graph without bucket build and gather; one whose lists are due (or fell short) the
    // full graph, as the host-driven step decides
    const bool keep = P.list_every > 1;
    const bool fresh = !keep || c->need_list || c->list_age >= P.list_every;
    StepGraph* sg = nullptr;
    for (StepGraph& g : c->step_graph)
        if (g.exec && g.pos == c->pos && g.kept == !fresh) sg = &g;
    if (!sg) {
        for (StepGraph& g : c->step_graph)
            if (!g.exec) { sg = &g; break; }
        if (!sg) return MPS_EDEVICE;   // a further buffer assignment: not expected
        const double4* start = c->pos;
        sg->kept = !fresh;
        rc = build_step_graph(c, sg);
        if (rc) {
            *sg = StepGraph{};   // the graph of the failed capture is left alone
            c->graphs_off = true;
            return rc;
        }
        sg->pos = start;
    }
    // ---- the control block of this step
    StepCtl& h = *c->ctl_host;
    // the skin of the lists this step uses: the adaptive one of a fresh gather, else the one
    // the kept lists were gathered with (no retry inside the graph: a kept step whose lists
    // fall short is taken again with fresh lists below)
    const double skin = fresh ? c->list_skin : c->gathered_skin;
    if (ppe) mixed_init_scalars(c, &h.cg_init);
    h.g[0] = P.g[0];
    h.g[1] = P.g[1];
    h.g[2] = c->dim == 3 ? P.g[2] : 0.0;
    h.half[0] = 0.5 * skin * re_max;
    h.half[1] = 0.5 * P.cell_skin * re_max;
    h.hv2[0] = make_radius(re_max * (1.0 + skin), c->band_x).hi;
    h.hv2[1] = make_radius(re_max * (1.0 + P.cell_skin), c->band_x).hi;
    h.can_retry = (fresh && skin < P.cell_skin) ? 1 : 0;
    h.attempt = 0;
    h.skin_err = 0;
    const int S = c->n_scenes;
    if (fresh && S > 1 && skin != c->rv_var_skin) {
        for (int s = 0; s < S; s++) {
            const SceneParams& sp = c->scn_host[(size_t)s];
            c->rv_var_host[s] = make_radius(std::max(sp.rn.re, sp.rl.re) * (1.0 + skin), c->band_x);
        }
        MPS_CUDA(c, cudaMemcpyAsync(c->rv_var, c->rv_var_host, sizeof(Radius) * (size_t)S,
                                    cudaMemcpyHostToDevice, c->stream));
        c->rv_var_skin = skin;
    }
    MPS_CUDA(c, cudaMemcpyAsync(c->ctl, c->ctl_host, sizeof(StepCtl), cudaMemcpyHostToDevice,
                                c->stream));
    if (fresh && (rc = bucket_order_word(c))) return rc;
    MPS_CUDA(c, cudaGraphLaunch(sg->exec, c->stream));
    state_ptrs_load(c, sg->after);
    if (fresh) c->order_valid = true;
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    // ---- what the step left
    const DevStatus& st = *c->st_host;
    const int attempts = h.attempt + 1;
    if (fresh) {
        const double used_skin = h.attempt ? P.cell_skin : skin;
        c->gathered_skin = used_skin;
        c->r_v = make_radius(re_max * (1.0 + used_skin), c->band_x);
        if (S > 1) c->scn_skin = used_skin;
        c->n_ghost_last = st.n_ghost;
    }
    rep->n_ghost = c->n_ghost_last;
    rep->n_surface = st.n_surface;
    rep->n_ppe_rows = st.n_ppe;
    double md;
    std::memcpy(&md, &st.max_disp_bits, sizeof md);
    rep->max_disp = std::sqrt(md);
    rep->cand_tests = (int64_t)st.cand_tests;
    rep->pairs_ppe = (int64_t)st.pairs_lap;
    rep->pairs_pnd = (int64_t)st.pairs_n;
    rep->list_tests = (int64_t)st.list_tests;
    rep->n0_pnd = c->n0_pnd;
    rep->n0_lap = c->n0_lap;
    rep->lambda = c->lambda;
    rep->cg_iters = rep->cg_outer = 0;
    rep->cg_resid = 0.0;
    rep->list_gathered = fresh ? 1 : 0;
    rep->step_graph = 1;
    rep->n_fast = 0;
    c->launches += sg->launches_pre + attempts * sg->launches_attempt;
    if (fresh) {
        bucket_branch_count(c, st);
        rep->bucket_merged = c->last_bucket_merged;
        rep->n_moved = (int64_t)st.n_mov;
        c->list_age = 0;
        c->need_list = false;
    } else {
        rep->bucket_merged = -1;
        rep->n_moved = 0;
    }
    if (st.err) {
        if (st.err & kErrNonfinite) return MPS_ENONFINITE;
        if (st.err & kErrCoincident) return MPS_ECOINCIDENT;
        if (st.err & kErrCap) return MPS_ECAP;
        return MPS_EDEVICE;
    }
    if (h.skin_err) {
        if (!fresh) {
            // the kept lists no longer cover the step (nothing was advanced): the step again
            // on lists gathered afresh
            c->need_list = true;
            return step_graph_step(c, rep);
        }
        if (S > 1) return MPS_ESKIN;
        // a particle outran the full skin: the host-driven step completes the lists of such
        // particles by a direct search (skinpatch.cu) and repeats the step (nothing advanced)
        c->force_host = true;
        rc = do_step(c, true, rep);
        c->force_host = false;
        return rc;
    }
    // next list skin: three times what this step's displacement needs, within
    // [kMinListSkin, cell_skin] (as the host-driven step)
    c->list_skin = std::min(P.cell_skin,
                            std::max(kMinListSkin, 3.0 * (2.0 * rep->max_disp / re_max) *
                                                       (keep ? P.list_every : 1)));
    c->launches += sg->launches_post;
    if (ppe) {
        const CgScalars& cg = *c->cg_host;
        c->launches += mixed_solve_launches(c, sg->guess, cg);
        rep->cg_iters = cg.total;
        rep->cg_outer = cg.outer;
        c->last_cg_iters = std::max(4, cg.total / std::max(cg.outer, 1));
        if (c->guess_m > 0) c->guess_n = std::min(c->guess_n + 1, c->guess_m);
        if (S == 1) {
            const double rel = cg.bb > 0.0 ? std::sqrt(cg.rr / cg.bb) : 0.0;
            rep->cg_resid = rel;
            c->scene_resid[0] = rel;
            if (!(cg.rr <= cg.ostop2)) return MPS_ECG_NOCONV;
        } else {
            double worst = 0.0;
            for (int k = 0; k < S; k++) {
                const double rr = c->scene_sums_host[2 * k], bb = c->scene_sums_host[2 * k + 1];
                const double rel = bb > 0.0 ? std::sqrt(rr / bb) : (rr > 0.0 ? HUGE_VAL : 0.0);
                c->scene_resid[(size_t)k] = (cg.outer > 0 || sg->guess) ? rel : 0.0;
                worst = std::max(worst, c->scene_resid[(size_t)k]);
            }
            rep->cg_resid = worst;
            if (!(worst <= P.cg_tol)) return MPS_ECG_NOCONV;
        }
    }
    if (keep) {
        // where r^{k+1} stands against r_b decides whether the next step may keep the lists
        c->list_age++;
        const double half = 0.5 * c->gathered_skin * re_max;
        double dn;
        std::memcpy(&dn, &st.max_disp_next_bits, sizeof dn);
        if (st.leave || std::sqrt(dn) > half) c->need_list = true;
    }
    c->steps_done++;
    rep->steps_done = c->steps_done;
    return MPS_OK;
}

}  // namespace mps
