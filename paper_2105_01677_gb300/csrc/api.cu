// api.cu -- the C ABI declared in include/mps.h: context set-up, the step driver and the
// host transfers.  Every stage of the step runs in this library's kernels; the host only
// sequences launches, polls the CG convergence flag and reads the status word.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ff.cuh"
#include "mps_internal.cuh"

namespace mps {

int cuda_fail(Ctx* c, cudaError_t e, const char* what) {
    if (c) {
        char buf[512];
        snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
        c->last_error = buf;
    }
    return MPS_EDEVICE;
}

void abort_capture(Ctx* c) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(c->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t tmp = nullptr;
        cudaStreamEndCapture(c->stream, &tmp);   // the captured-into graph or null: not used
    }
    cudaGetLastError();
}

namespace {

struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Reference density and lambda of an ideal lattice (Eq. 5; lambda of Eq. 7): every integer
// offset o != 0 with |o| l0 < re contributes w(|o| l0) — re/r - 1 (Eq. 4), or (1 - r/re)^3
// for kernel 1 — and w |o|^2 l0^2 to lambda.
void lattice_constants(int dim, double l0, double re, double* n0, double* lambda, int* count,
                       int kernel = 0) {
    const int m = (int)std::ceil(re / l0) + 1;
    const int mz = dim == 3 ? m : 0;
    double sw = 0.0, swr2 = 0.0;
    int cnt = 0;
    for (int c = -mz; c <= mz; c++)
        for (int b = -m; b <= m; b++)
            for (int a = -m; a <= m; a++) {
                const int k = a * a + b * b + c * c;
                if (k == 0) continue;
                const double r = l0 * std::sqrt((double)k);
                if (!(r < re)) continue;
                const double t = 1.0 - r / re;
                const double w = kernel == 1 ? t * t * t : re / r - 1.0;
                sw += w;
                swr2 += w * r * r;
                cnt++;
            }
    *n0 = sw;
    *lambda = sw > 0.0 ? swr2 / sw : 0.0;
    *count = cnt;
}

}  // namespace

// FP32 pre-filter band for r^2 < re^2 (see gather.cu).  Coordinates are stored relative to
// the grid origin, so |x| <= X; each is rounded once to FP32 (error <= 2^-24 X), the
// difference and the squares add a few more roundings.
Radius make_radius(double re, double X) {
    Radius r;
    r.re = re;
    r.re2 = re * re;
    r.re_f = (float)re;
    const double E = std::ldexp(X, -23);
    const double delta = 2.0 * E + std::ldexp(re, -22);
    const double eps = 2.0 * (3.0 * delta * (2.0 * re + delta)) + std::ldexp(re * re, -19);
    r.lo = std::nextafter((float)(r.re2 - eps), 0.0f);
    r.hi = std::nextafter((float)(r.re2 + eps), INFINITY);
    if (!(r.lo > 0.0f)) r.lo = 0.0f;
    // float-float tier: coordinates split into hi + lo floats carry ~2^-48 X of error, the
    // float-float squares and sums ~2^-46 relative; the binary64 evaluation it must agree
    // with rounds at 2^-53.  Pairs closer to the cutoff than this go to binary64.
    r.re2_h = (float)r.re2;
    r.re2_l = (float)(r.re2 - (double)r.re2_h);
    r.re_l = (float)(re - (double)r.re_f);
    r.inv_re = 1.0 / re;
    r.inv_f = (float)r.inv_re;
    r.inv_l = (float)(r.inv_re - (double)r.inv_f);
    const double tol = 8.0 * (2.0 * re * std::sqrt(3.0) * std::ldexp(X, -46)) +
                       8.0 * std::ldexp(re * re, -45);
    r.ff_tol = (float)tol;
    return r;
}

namespace {

int round_up(int v, int m) { return (v + m - 1) / m * m; }

template <class T>
int alloc_dev(Ctx* c, T** out, size_t count) {
    size_t bytes = std::max<size_t>(count * sizeof(T), 256);
    void* p = nullptr;
    if (c->prm.alloc) {
        p = c->prm.alloc(bytes, c->prm.alloc_user);
        if (!p) return MPS_ENOMEM;
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->last_error = "cudaMalloc failed";
            return MPS_ENOMEM;
        }
    }
    c->allocations.push_back(p);
    *out = (T*)p;
    return MPS_OK;
}

void free_all(Ctx* c) {
    for (void* p : c->allocations) {
        if (c->prm.alloc && c->prm.release) c->prm.release(p, c->prm.alloc_user);
        else if (!c->prm.alloc) cudaFree(p);
    }
    c->allocations.clear();
}

void free_one(Ctx* c, void* p) {
    auto it = std::find(c->allocations.begin(), c->allocations.end(), p);
    if (it == c->allocations.end()) return;
    c->allocations.erase(it);
    if (c->prm.alloc && c->prm.release) c->prm.release(p, c->prm.alloc_user);
    else if (!c->prm.alloc) cudaFree(p);
}

int check_params(const mps_params* P) {
    if (!P) return MPS_EINVAL;
    if (P->dim != 2 && P->dim != 3) return MPS_EINVAL;
    if (!(P->l0 > 0) || !(P->re_n > 0) || !(P->re_lap > 0) || !(P->rho > 0) || !(P->dt > 0))
        return MPS_EINVAL;
    if (!(P->nu >= 0) || !(P->beta >= 0) || !(P->cell_skin >= 0) || !(P->alpha_c >= 0))
        return MPS_EINVAL;
    if (P->pressure_mode != 0 && P->pressure_mode != 1) return MPS_EINVAL;
    if (P->precision != 0 && P->precision != 1) return MPS_EINVAL;
    if (P->pressure_mode == 0 && !(P->cg_tol > 0)) return MPS_EINVAL;
    if (P->pressure_mode == 1 && !(P->gamma > 0)) return MPS_EINVAL;
    if ((P->alloc == nullptr) != (P->release == nullptr)) return MPS_EINVAL;
    if (P->list_every < 0) return MPS_EINVAL;
    if (P->ppe_host_loop != 0 && P->ppe_host_loop != 1) return MPS_EINVAL;
    if (P->cg_x0 < 0 || P->cg_x0 > 4) return MPS_EINVAL;
    if (P->inner_cg < 0 || P->inner_cg > 1) return MPS_EINVAL;
    if (P->spmv_block != 0 && P->spmv_block != 256 && P->spmv_block != 512) return MPS_EINVAL;
    if (P->build_block != 0 && P->build_block != 64 && P->build_block != 128 &&
        P->build_block != 256)
        return MPS_EINVAL;
    if (P->bucket_sort != 0 && P->bucket_sort != 1) return MPS_EINVAL;
    if (P->step_graph < 0 || P->step_graph > 2) return MPS_EINVAL;
    if (P->cg_unroll != 0 && P->cg_unroll != 1 && P->cg_unroll != 2 && P->cg_unroll != 4)
        return MPS_EINVAL;
    if (P->predict_tpr != 0 && P->predict_tpr != 1 && P->predict_tpr != 2 && P->predict_tpr != 4)
        return MPS_EINVAL;
    if (P->kernel < 0 || P->kernel > 1 || P->gradient_form < 0 || P->gradient_form > 1 ||
        P->source_term < 0 || P->source_term > 2 || (P->source_term >= 1 && P->kernel != 0))
        return MPS_EINVAL;
    // the matrix-free FP32 operator recomputes the coefficients of Eq. 4's kernel only
    if (P->pressure_mode == 0 && P->precision == 1 && P->ppe_operator == 1 && P->kernel != 0)
        return MPS_EINVAL;
    if (P->gather_block != 0 && P->gather_block != 32 && P->gather_block != 64 &&
        P->gather_block != 96 && P->gather_block != 128)
        return MPS_EINVAL;
    for (int a = 0; a < P->dim; a++)
        if (!(P->box_max[a] > P->box_min[a]) || !std::isfinite(P->box_min[a]) ||
            !std::isfinite(P->box_max[a]))
            return MPS_EINVAL;
    return MPS_OK;
}

int check_host_state(int64_t n, int dim, const double* pos, const double* vel, const int8_t* types) {
    for (int64_t k = 0; k < n * dim; k++) {
        if (pos && !std::isfinite(pos[k])) return MPS_ENONFINITE;
        if (vel && !std::isfinite(vel[k])) return MPS_ENONFINITE;
    }
    if (types)
        for (int64_t i = 0; i < n; i++)
            if (types[i] < MPS_FLUID || types[i] > MPS_GHOST) return MPS_EINVAL;
    return MPS_OK;
}

// Constants of one scene with spacing l0 (the radii scale with it) and its own grid box.
int scene_constants(const mps_params& P, double l0, const double* bmin, const double* bmax,
                    SceneParams* sp, int* cnt_n, int* cnt_l, int* cnt_h) {
    const int dim = P.dim;
    const double re_n = P.re_n / P.l0 * l0, re_lap = P.re_lap / P.l0 * l0;
    double lam_n, lam, n0h, lamh;
    lattice_constants(dim, l0, re_n, &sp->n0_pnd, &lam_n, cnt_n, P.kernel);
    lattice_constants(dim, l0, re_lap, &sp->n0_lap, &lam, cnt_l, P.kernel);
    if (!(sp->n0_pnd > 0) || !(sp->n0_lap > 0)) return MPS_EINVAL;
    sp->lambda = lam;
    sp->coef_lap = (2.0 * dim) / (sp->n0_lap * lam);
    sp->coef_ppe = (2.0 * dim) / (sp->n0_lap * lam * P.rho);
    sp->coef_grad = (double)dim / sp->n0_pnd;
    sp->own_h = std::max(re_n, re_lap) * (1.0 + P.cell_skin);
    lattice_constants(dim, l0, sp->own_h, &n0h, &lamh, cnt_h);
    for (int a = 0; a < 3; a++) {
        if (a < dim) {
            if (!(bmax[a] > bmin[a]) || !std::isfinite(bmin[a]) || !std::isfinite(bmax[a]))
                return MPS_EINVAL;
            sp->own_bmin[a] = bmin[a];
            const double q = std::floor((bmax[a] - bmin[a]) / sp->own_h) + 1.0;
            if (q > 16384.0) return MPS_EINVAL;
            sp->own_ncell[a] = (int)q;
        } else {
            sp->own_bmin[a] = 0.0;
            sp->own_ncell[a] = 1;
        }
    }
    sp->rn.re = re_n;    // completed with the bands once the shared grid is known
    sp->rl.re = re_lap;
    sp->pad = 0;
    return MPS_OK;
}

int setup(Ctx* c, const mps_scene* scenes, int n_scenes) {
    const mps_params& P = c->prm;
    const int dim = P.dim;
    c->dim = dim;
    c->n_scenes = n_scenes;
    c->scn_host.assign((size_t)n_scenes, SceneParams{});
    int cnt_n = 0, cnt_l = 0, cnt_h = 0, rc;
    for (int s = 0; s < n_scenes; s++) {
        const double l0 = scenes ? scenes[s].l0 : P.l0;
        if (!(l0 > 0) || !std::isfinite(l0)) return MPS_EINVAL;
        if ((rc = scene_constants(P, l0, scenes ? scenes[s].box_min : P.box_min,
                                  scenes ? scenes[s].box_max : P.box_max, &c->scn_host[s], &cnt_n,
                                  &cnt_l, &cnt_h)))
            return rc;
    }
    // list caps: the neighbour counts depend only on the radii in units of l0 (the same for
    // every scene)
    c->cap = P.nbr_cap > 0 ? round_up(P.nbr_cap, 32) : round_up((int)std::ceil(1.5 * cnt_l), 32);
    c->cap_n = round_up(std::max((int)std::ceil(1.5 * cnt_n),
                                 (int)std::ceil((double)c->cap * cnt_n / std::max(cnt_l, 1))), 32);
    // candidate lists hold every kind within h = max(re)(1 + s): sized from the
    // ideal-lattice count within h, scaled like the neighbour cap
    c->cap_v = round_up(std::max((int)std::ceil(1.5 * cnt_h),
                                 (int)std::ceil((double)c->cap * cnt_h / std::max(cnt_l, 1))), 32);
    // at least one SELL slot group per list (a radius below l0 has no lattice neighbours)
    c->cap = std::max(c->cap, 32);
    c->cap_n = std::max(c->cap_n, 32);
    c->cap_v = std::max(c->cap_v, 32);
    // shared grid: cells of the largest scene's side, covering every scene's own grid
    GridDesc& g = c->grid;
    g.dim = dim;
    double hmax = 0.0, skin_half = 1e300, re_skin = 1e300;
    for (const SceneParams& sp : c->scn_host) {
        hmax = std::max(hmax, sp.own_h);
        skin_half = std::min(skin_half, 0.5 * P.cell_skin * std::max(sp.rn.re, sp.rl.re));
        re_skin = std::min(re_skin, std::max(sp.rn.re, sp.rl.re));
    }
    c->h = hmax;
    c->skin_half = skin_half;
    c->re_skin = re_skin;
    g.h = hmax;
    g.inv_h = 1.0 / hmax;
    g.inv_hf = (float)g.inv_h;
    int maxc = 1;
    double X = 0.0;
    for (int a = 0; a < 3; a++) {
        if (a < dim) {
            // one scene: its own grid; an ensemble: enough cells of the largest side to cover
            // every scene's own grid (each scene's own grid still decides its GHOSTs)
            double lo = 1e300, hi = -1e300;
            for (const SceneParams& sp : c->scn_host) {
                lo = std::min(lo, sp.own_bmin[a]);
                hi = std::max(hi, sp.own_bmin[a] + sp.own_ncell[a] * sp.own_h);
            }
            g.bmin[a] = lo;
            const double q = n_scenes == 1 ? (double)c->scn_host[0].own_ncell[a]
                                           : std::max(1.0, std::ceil((hi - lo) / hmax));
            if (q > 16384.0) return MPS_EINVAL;
            g.ncell[a] = (int)q;
            maxc = std::max(maxc, g.ncell[a]);
            X = std::max(X, (q + 1.0) * hmax);
        } else {
            g.bmin[a] = 0.0;
            g.ncell[a] = 1;
        }
    }
    int bits = 1;
    while ((1 << bits) < maxc) bits++;
    int sbits = 0;
    while ((1 << sbits) < n_scenes + 1) sbits++;
    if (dim * bits > 28 || dim * bits + sbits > 31) return MPS_EINVAL;
    g.bits = bits;
    c->scene_shift = (uint32_t)(dim * bits);
    g.ghost_key = (uint32_t)n_scenes << c->scene_shift;
    c->ntable = (int64_t)n_scenes << c->scene_shift;
    c->sort_bits = dim * bits + sbits;
    for (SceneParams& sp : c->scn_host) {
        const double re_n = sp.rn.re, re_lap = sp.rl.re;
        sp.rn = make_radius(re_n, X);
        sp.rl = make_radius(re_lap, X);
        sp.rv = make_radius(sp.own_h, X);
        const ff cre = ff_from_double(sp.coef_ppe * re_lap), nco = ff_from_double(-sp.coef_ppe);
        sp.cre_h = cre.h;
        sp.cre_l = cre.l;
        sp.ncoef_h = nco.h;
        sp.ncoef_l = nco.l;
        const ff cre2 = ff_from_double(sp.coef_lap * re_lap), nco2 = ff_from_double(-sp.coef_lap);
        sp.cre2_h = cre2.h;
        sp.cre2_l = cre2.l;
        sp.ncoef2_h = nco2.h;
        sp.ncoef2_l = nco2.l;
    }
    // scene 0 also in scalars (the single-scene kernels take their constants from these)
    const SceneParams& s0 = c->scn_host[0];
    c->n0_pnd = s0.n0_pnd;
    c->n0_lap = s0.n0_lap;
    c->lambda = s0.lambda;
    c->coef_lap = s0.coef_lap;
    c->coef_ppe = s0.coef_ppe;
    c->coef_grad = s0.coef_grad;
    c->inv_dt2 = 1.0 / (P.dt * P.dt);
    c->diag_add = P.alpha_c / (P.dt * P.dt);
    c->r_n = s0.rn;
    c->r_lap = s0.rl;
    c->r_v = make_radius(c->h, X);
    c->band_x = X;
    c->list_skin = P.cell_skin;
    c->scene_resid.assign((size_t)n_scenes, 0.0);
    return MPS_OK;
}

int allocate(Ctx* c) {
    const size_t n = (size_t)c->n;
    int rc = 0;
#define A(ptr, count) \
    if ((rc = alloc_dev(c, &c->ptr, (count)))) return rc;
    const size_t sv = sell_size(c->n, c->cap_v), sl = sell_size(c->n, c->cap),
                 sn = sell_size(c->n, c->cap_n);
    A(pos, n) A(vel, n) A(pos_alt, n) A(vel_alt, n) A(type, n) A(type_alt, n) A(id, n) A(id_alt, n)
    A(p, n) A(p_alt, n) A(pos32, n) A(pos32lo, n) A(pos_star, n) A(vel_star, n) A(pos32_star, n)
    A(pff_star, 2 * n) A(nstar, n) A(flag, n) A(bvec, n) A(diag, n) A(diag32, n) A(phat, n)
    A(vl_col, sv) A(vl_cnt, n) A(vel32, n)
    // nb_lap_col also stages the number-density entries of a row while it is assembled
    A(nb_n_col, sn) A(nb_n_cnt, n) A(nb_lap_cnt, n) A(nb_lap_col, sl)
    if (c->prm.pressure_mode == 0) {
        if (c->prm.precision == 1) {
            A(nb_lap_v32, sl) A(nb_lap_vlo, sl)
            A(cg_r32, n) A(cg_d32, n) A(cg_q32, n) A(cg_x32, n) A(cg_xhl, n) A(cg_s32, n)
        } else {
            A(nb_lap_v64, sl)
        }
        A(cg_r, n) A(cg_d, n) A(cg_q, n)
        // the guess history: the last cg_x0 solutions (none valid yet)
        c->guess_m = std::min(c->prm.cg_x0, Ctx::kGuessMax);
        c->guess_n = 0;
        for (int k = 0; k < c->guess_m; k++) {
            A(ph[k], n) A(ph_alt[k], n)
            MPS_CUDA(c, cudaMemsetAsync(c->ph[k], 0, n * sizeof(double), c->stream));
        }
    }
    if (c->prm.list_every > 1) A(pos_b, n)
    A(scn, (size_t)c->n_scenes) A(scene_sums, 2 * (size_t)c->n_scenes)
    if (c->n_scenes > 1) { A(sid, n) A(sid_id, n) }
    if (c->prm.pressure_mode == 0 && c->prm.source_term == 2) { A(ecs_nk, n) A(ecs_dk, n) }
    c->cap_v_alloc = c->cap_v;
    c->ntable_alloc = c->ntable;
    A(key, n) A(key_alt, n) A(perm, n) A(perm_alt, n)
    const int64_t tiles = ((int64_t)n + 2047) / 2048;
    A(hist, 256 * tiles) A(hist_scan, 256 * tiles)
    A(cell_count, c->ntable) A(cell_start, c->ntable + 1) A(occ, n + 1)
    c->mov_cap = (int)std::min<size_t>(n, 16384);
    A(mvf, n) A(mov_key, c->mov_cap) A(mov_slot, c->mov_cap) A(mov_cnt, 4 * (size_t)c->mov_cap)
    A(mov_by_slot, c->mov_cap) A(mov_by_key, c->mov_cap) A(order_ok, 1)
    A(mark_f, n + 1) A(mark_fw, n + 1) A(scan_f, n + 1) A(scan_fw, n + 1) A(rows_f, n) A(rows_fw, n)
    const int64_t sw = std::max(std::max(scan_scratch_words(256 * tiles), scan_scratch_words(c->ntable + 1)),
                                scan_scratch_words((int64_t)n + 1));
    A(scan_scratch, sw)
    A(partials, 4096) A(cg, 1) A(st, 1)
    A(fast_idx, (size_t)skin_patch_cap(c))
    c->stage_bytes = n * (3 * 8 * 2 + 8 + 8 + 4 + 2) + 1024;
    { uint8_t* s8 = nullptr; if ((rc = alloc_dev(c, &s8, c->stage_bytes))) return rc; c->stage = s8; }
#undef A
    if (cudaMallocHost(&c->st_host, sizeof(DevStatus)) != cudaSuccess) return MPS_ENOMEM;
    if (cudaMallocHost(&c->cg_host, sizeof(CgScalars)) != cudaSuccess) return MPS_ENOMEM;
    MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
    MPS_CUDA(c, cudaMemsetAsync(c->cg, 0, sizeof(CgScalars), c->stream));
    MPS_CUDA(c, cudaMemsetAsync(c->nb_lap_cnt, 0, n * sizeof(int32_t), c->stream));
    MPS_CUDA(c, cudaMemsetAsync(c->nb_n_cnt, 0, n * sizeof(int32_t), c->stream));
    MPS_CUDA(c, cudaMemsetAsync(c->phat, 0, n * sizeof(double), c->stream));
    MPS_CUDA(c, cudaMemcpyAsync(c->scn, c->scn_host.data(), sizeof(SceneParams) * c->scn_host.size(),
                                cudaMemcpyHostToDevice, c->stream));
    return MPS_OK;
}

// The grid of another cell skin s (the tuner's choice of the cell side h = max(re)(1 + s)):
// cells per axis, Morton bits, the cell table, the FP32 bands and the candidate-list capacity
// are derived again; the cell table, its scan scratch and the candidate lists are allocated
// again when they grow.  The state keeps its slot order; the next bucket build sorts it into
// the new cells and the next step gathers its lists afresh.  On failure the previous grid
// stays in force.
int regrid(Ctx* c, double skin) {
    if (skin == c->prm.cell_skin) return MPS_OK;
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));   // nothing in flight on the old buffers
    const double old_skin = c->prm.cell_skin, list_skin = c->list_skin;
    const mps_scene* sc = c->n_scenes > 1 ? c->scenes_host.data() : nullptr;
    auto restore = [&](int rc) {
        c->prm.cell_skin = old_skin;
        setup(c, sc, c->n_scenes);   // the derivation that succeeded before
        c->list_skin = list_skin;
        return rc;
    };
    c->prm.cell_skin = skin;
    int rc = setup(c, sc, c->n_scenes);
    if (rc) return restore(rc);
    // smaller cells need no fewer candidate slots than the lists already have: keep the
    // allocated capacity (headroom for compressed regions at no cost)
    c->cap_v = std::max(c->cap_v, c->cap_v_alloc);
    int32_t* vl_col = nullptr;
    uint32_t *cell_count = nullptr, *scan_scratch = nullptr;
    int32_t* cell_start = nullptr;
    const size_t n = (size_t)c->n;
    if (c->cap_v > c->cap_v_alloc &&
        (rc = alloc_dev(c, &vl_col, sell_size(c->n, c->cap_v))))
        return restore(rc);
    if (c->ntable > c->ntable_alloc) {
        const int64_t tiles = ((int64_t)n + 2047) / 2048;
        const int64_t sw = std::max(std::max(scan_scratch_words(256 * tiles),
                                             scan_scratch_words(c->ntable + 1)),
                                    scan_scratch_words((int64_t)n + 1));
        if ((rc = alloc_dev(c, &cell_count, (size_t)c->ntable)) ||
            (rc = alloc_dev(c, &cell_start, (size_t)c->ntable + 1)) ||
            (rc = alloc_dev(c, &scan_scratch, (size_t)sw))) {
            free_one(c, vl_col);
            free_one(c, cell_count);
            free_one(c, cell_start);
            return restore(rc);
        }
    }
    // the graphs captured the old grid (keys, table size, sort passes) and buffers
    bucket_graphs_destroy(c);
    step_graphs_destroy(c);
    if (vl_col) {
        free_one(c, c->vl_col);
        c->vl_col = vl_col;
        c->cap_v_alloc = c->cap_v;
    }
    if (cell_count) {
        free_one(c, c->cell_count);
        free_one(c, c->cell_start);
        free_one(c, c->scan_scratch);
        c->cell_count = cell_count;
        c->cell_start = cell_start;
        c->scan_scratch = scan_scratch;
        c->ntable_alloc = c->ntable;
    }
    c->list_skin = std::min(list_skin, skin);
    c->scn_skin = -1.0;
    c->need_list = true;
    c->order_valid = false;   // keys of another grid
    MPS_CUDA(c, cudaMemcpyAsync(c->scn, c->scn_host.data(), sizeof(SceneParams) * c->scn_host.size(),
                                cudaMemcpyHostToDevice, c->stream));
    if (c->rv_var) {
        // the step graph's table of candidate radii: the full-skin half follows s, the
        // adaptive half is written again before the next graph step
        const size_t S = (size_t)c->n_scenes;
        for (size_t k = 0; k < S; k++) {
            const SceneParams& sp = c->scn_host[k];
            c->rv_var_host[S + k] =
                make_radius(std::max(sp.rn.re, sp.rl.re) * (1.0 + skin), c->band_x);
        }
        MPS_CUDA(c, cudaMemcpyAsync(c->rv_var + S, c->rv_var_host + S, sizeof(Radius) * S,
                                    cudaMemcpyHostToDevice, c->stream));
        c->rv_var_skin = -1.0;
    }
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    return MPS_OK;
}

// Host data -> device staging (original order) -> state arrays (slot = id).
int read_status(Ctx* c);

// validate: check the staged values on the device first (mps_write_state); the context's
// state is replaced only if they are finite and of known kinds
// device: the caller's arrays are in device memory (copies device to device)
int upload_state(Ctx* c, const double* pos, const double* vel, const int8_t* types, bool have_state,
                 bool validate = false, bool device = false) {
    const cudaMemcpyKind in = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t n = (size_t)c->n, dim = (size_t)c->dim;
    int rc_check;
    uint8_t* base = (uint8_t*)c->stage;
    double* d_pos = (double*)base;
    double* d_vel = d_pos + n * dim;
    int8_t* d_t = (int8_t*)(d_vel + n * dim);
    if (have_state && (!vel || !types)) {
        // keep the current velocities / kinds: bring them to original order first
        launch_unpermute(c, nullptr, vel ? nullptr : d_vel, nullptr, nullptr, nullptr,
                         types ? nullptr : d_t);
    }
    MPS_CUDA(c, cudaMemcpyAsync(d_pos, pos, n * dim * sizeof(double), in, c->stream));
    if (vel) MPS_CUDA(c, cudaMemcpyAsync(d_vel, vel, n * dim * sizeof(double), in, c->stream));
    else if (!have_state) MPS_CUDA(c, cudaMemsetAsync(d_vel, 0, n * dim * sizeof(double), c->stream));
    if (types) MPS_CUDA(c, cudaMemcpyAsync(d_t, types, n, in, c->stream));
    if (validate) {
        MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
        launch_check_stage(c, d_pos, vel ? d_vel : nullptr, types ? d_t : nullptr);
        launch_same_state(c, d_pos, vel ? d_vel : nullptr, types ? d_t : nullptr);
        if ((rc_check = read_status(c))) return rc_check;
        if (c->st_host->err & kErrNonfinite) return MPS_ENONFINITE;
        if (c->st_host->err & kErrKind) return MPS_EINVAL;
        // the state the context already holds, bit for bit: nothing to replace (its lists,
        // the PPE guess history, p, n* and the flags stay as the last step left them)
        if (!c->st_host->differs) return MPS_OK;
    }
    c->need_list = true;
    c->order_valid = false;   // slot = id: the next bucket build sorts from scratch
    launch_ingest(c, d_pos, d_vel, d_t, false, false);
    launch_gather_props(c);   // slot = id again
    c->guess_n = 0;   // a written state starts its solve from zero
    MPS_CUDA(c, cudaGetLastError());
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    return MPS_OK;
}

int read_status(Ctx* c) {
    MPS_CUDA(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    bucket_branch_count(c, *c->st_host);
    return MPS_OK;
}

int status_error(const DevStatus& s) {
    if (s.err & kErrNonfinite) return MPS_ENONFINITE;
    if (s.err & kErrCoincident) return MPS_ECOINCIDENT;
    if (s.err & kErrCap) return MPS_ECAP;
    if (s.err & kErrWait) return MPS_EDEVICE;
    return MPS_OK;
}

double bits_to_double(unsigned long long b) {
    double d;
    std::memcpy(&d, &b, sizeof d);
    return d;
}

void stage_begin(Ctx* c, int s) {
    if (c->profiling) cudaEventRecord(c->ev[2 * s], c->stream);
}
void stage_end(Ctx* c, int s) {
    if (c->profiling) cudaEventRecord(c->ev[2 * s + 1], c->stream);
}
// after a stream sync: add the elapsed time of every stage recorded in this step
void stage_collect(Ctx* c, const bool* used) {
    if (!c->profiling) return;
    for (int s = 0; s < MPS_NSTAGES; s++) {
        if (!used[s]) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev[2 * s], c->ev[2 * s + 1]) == cudaSuccess) {
            c->stage_ms[s] += ms;
            c->stage_calls[s] += 1;
        }
    }
}


// Candidate lists of the next gather within max(re)(1 + skin) of every scene, with the FP32
// bands of the grid in force.
int set_candidate_radius(Ctx* c, double skin) {
    c->gathered_skin = skin;
    if (c->n_scenes == 1) {
        c->r_v = make_radius(c->re_skin * (1.0 + skin), c->band_x);
    } else if (skin != c->scn_skin) {
        for (SceneParams& sp : c->scn_host)
            sp.rv = make_radius(std::max(sp.rn.re, sp.rl.re) * (1.0 + skin), c->band_x);
        MPS_CUDA(c, cudaMemcpyAsync(c->scn, c->scn_host.data(),
                                    sizeof(SceneParams) * c->scn_host.size(),
                                    cudaMemcpyHostToDevice, c->stream));
        c->scn_skin = skin;
    }
    return MPS_OK;
}
}  // namespace

// One step (advance) or steps 1-5 only (solve).

int do_step(Ctx* c, bool advance, mps_report* rep) {
    const mps_params& P = c->prm;
    int rc;
    if (step_graph_eligible(c, advance)) return step_graph_step(c, rep);
    rep->step_graph = 0;
    rep->n_fast = 0;
    const bool keep = P.list_every > 1;
    // the radius the skin is measured against: max(re) (of the scene with the smallest
    // spacing in an ensemble)
    const double re_max = c->re_skin;
    // Candidate lists are gathered within the skin the recent motion needs over the lists'
    // lifetime (the grid's cells keep the full skin); a step whose motion exceeds the skin
    // of the lists in use is gathered again (with the full skin if a fresh gather already
    // fell short), so the sets stay exact.  In an ensemble every scene's candidate radius
    // is its own max(re) times (1 + that skin).
    const bool adapt = true;
    const size_t n = (size_t)c->n;
    // Candidate lists are gathered at r_b and serve while every particle stays within
    // s max(re)/2 of r_b: a pair closer than re at r^k or r* is then closer than h at r_b.
    // A kept list that fails the check for r* is gathered afresh at r^k and the step
    // restarts (r^k, u^k are untouched until the update).
    bool fresh = !keep || c->need_list || c->list_age >= P.list_every;
    // particles beyond the full skin: their pairs found by a direct search at r* (one scene)
    bool patch = false, patched = false;
    for (;;) {
        MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
        if (fresh) {
            stage_begin(c, MPS_STAGE_BUCKET);
            if ((rc = bucket_build(c, true))) return rc;               // 1
            stage_end(c, MPS_STAGE_BUCKET);
            if (keep)
                MPS_CUDA(c, cudaMemcpyAsync(c->pos_b, c->pos, n * sizeof(double4),
                                            cudaMemcpyDeviceToDevice, c->stream));
        }
        if (!fresh) launch_copy_state_star(c);   // a build's permutation writes r* := r itself
        if (fresh) {
            if ((rc = set_candidate_radius(c, adapt ? c->list_skin : P.cell_skin))) return rc;
            MPS_CUDA(c, cudaMemsetAsync(c->vl_cnt, 0, n * sizeof(int32_t), c->stream));
            stage_begin(c, MPS_STAGE_GATHER);
            launch_verlet(c);                                          // candidates at r_b = r^k
            stage_end(c, MPS_STAGE_GATHER);
        }
        stage_begin(c, MPS_STAGE_PREDICT);
        launch_predict_rows(c);                                        // 2
        if (P.pressure_mode == 0 && P.source_term == 2) launch_ecs_rates(c);   // at r^k, u^k
        stage_end(c, MPS_STAGE_PREDICT);
        if (patch) {
            launch_fast_mark(c, 0.5 * P.cell_skin * re_max);
            if ((rc = read_status(c))) return rc;
            const int n_fast = (int)c->st_host->n_fast;
            rep->n_fast = n_fast;
            if (n_fast > skin_patch_cap(c)) return MPS_ESKIN;
            if ((rc = launch_fast_patch(c, n_fast, c->r_v.hi))) return rc;
            patched = true;
        }
        // per-slot outputs of the build; slots it does not visit (GHOST) keep these zeros
        launch_clear_rows(c);
        stage_begin(c, MPS_STAGE_BUILD);
        launch_build_rows(c);                                          // 3 (+ 4 for the EOS)
        stage_end(c, MPS_STAGE_BUILD);
        MPS_CUDA(c, cudaGetLastError());
        if ((rc = read_status(c))) return rc;
        const DevStatus& s = *c->st_host;
        if (fresh) c->n_ghost_last = s.n_ghost;
        rep->n_ghost = c->n_ghost_last;
        rep->bucket_merged = fresh ? c->last_bucket_merged : -1;
        rep->n_moved = fresh ? (int64_t)s.n_mov : 0;
        rep->n_surface = s.n_surface;
        rep->n_ppe_rows = s.n_ppe;
        rep->max_disp = std::sqrt(bits_to_double(s.max_disp_bits));   // device keeps the square
        rep->cand_tests = (int64_t)s.cand_tests;
        rep->pairs_ppe = (int64_t)s.pairs_lap;
        rep->pairs_pnd = (int64_t)s.pairs_n;
        rep->list_tests = (int64_t)s.list_tests;
        rep->n0_pnd = c->n0_pnd;
        rep->n0_lap = c->n0_lap;
        rep->lambda = c->lambda;
        rep->cg_iters = rep->cg_outer = 0;
        rep->cg_resid = 0.0;
        rep->list_gathered = fresh ? 1 : 0;
        if ((rc = status_error(s))) return rc;
        const double half = adapt ? 0.5 * c->gathered_skin * re_max : c->skin_half;
        if (rep->max_disp > half && !patched) {
            if (!fresh) {                                              // a kept list falls short
                fresh = true;                                          // gather afresh at r^k
                continue;
            }
            if (adapt && c->gathered_skin < P.cell_skin) {
                c->list_skin = P.cell_skin;                            // the full skin
                continue;
            }
            if (c->n_scenes == 1) {                                    // complete the lists of
                patch = true;                                          // the particles beyond it
                continue;
            }
            return MPS_ESKIN;
        }
        break;
    }
    if (adapt) {
        // next list skin: three times what the motion of the lists' lifetime needs at this
        // step's displacement, within [kMinListSkin, cell_skin]
        const double need = 2.0 * rep->max_disp / re_max * (keep ? P.list_every : 1);
        c->list_skin = std::min(P.cell_skin, std::max(kMinListSkin, 3.0 * need));
    }
    if (fresh) {
        c->list_age = 0;
        c->need_list = false;
    }
    bool used[MPS_NSTAGES] = {fresh, fresh, true, true, P.pressure_mode == 0, true};
    if (P.pressure_mode == 0) {                                    // 4, 5
        stage_begin(c, MPS_STAGE_PPE);
        if ((rc = ppe_solve(c, rep))) return rc;
        if (c->guess_m > 0) {
            // the next solve starts from this one (and the ones before it): shift the history
            launch_push_history(c);
            c->guess_n = std::min(c->guess_n + 1, c->guess_m);
        }
        stage_end(c, MPS_STAGE_PPE);
    }
    stage_begin(c, MPS_STAGE_UPDATE);
    if (c->vjp && P.pressure_mode == 0)   // the reverse step needs p before the clamp
        MPS_CUDA(c, cudaMemcpyAsync(c->adj.ppre, c->p, n * sizeof(double),
                                    cudaMemcpyDeviceToDevice, c->stream));
    if ((rc = launch_pressure_floor(c))) return rc;
    if (advance) launch_gradient_correct(c);                       // 6
    stage_end(c, MPS_STAGE_UPDATE);
    MPS_CUDA(c, cudaGetLastError());
    if (keep && advance) {
        // where r^{k+1} stands against r_b decides whether the next step may keep the lists
        MPS_CUDA(c, cudaMemcpyAsync(c->st_host, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                                    c->stream));
    }
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    stage_collect(c, used);
    if (keep && advance) {
        const DevStatus& s = *c->st_host;
        c->list_age++;
        const double half = adapt ? 0.5 * c->gathered_skin * re_max : c->skin_half;
        if (s.leave || std::sqrt(bits_to_double(s.max_disp_next_bits)) > half) c->need_list = true;
    }
    if (advance) c->steps_done++;
    rep->steps_done = c->steps_done;
    return MPS_OK;
}

namespace {
int alloc_adjoint(Ctx* c) {
    AdjBuffers& a = c->adj;
    if (a.ready) return MPS_OK;
    const size_t n = (size_t)c->n;
    int rc;
    if ((rc = alloc_dev(c, &a.gr, n)) || (rc = alloc_dev(c, &a.gu, n)) ||
        (rc = alloc_dev(c, &a.gG, n)) || (rc = alloc_dev(c, &a.grs, n)) ||
        (rc = alloc_dev(c, &a.gus, n)) || (rc = alloc_dev(c, &a.out_r, n)) ||
        (rc = alloc_dev(c, &a.out_u, n)) || (rc = alloc_dev(c, &a.gphat, n)) ||
        (rc = alloc_dev(c, &a.pbar, n)) || (rc = alloc_dev(c, &a.lam, n)) ||
        (rc = alloc_dev(c, &a.gn, n)) || (rc = alloc_dev(c, &a.ppre, n)) ||
        (rc = alloc_dev(c, &a.amin, n)) || (rc = alloc_dev(c, &a.was_ghost, n)) ||
        (rc = alloc_dev(c, &a.gsum, 4)) || (rc = alloc_dev(c, &a.gnu, n))) {
        // all or none: hand back what was taken, so that a retry starts clean
        void* bufs[] = {a.gr, a.gu, a.gG, a.grs, a.gus, a.out_r, a.out_u, a.gphat, a.pbar,
                        a.lam, a.gn, a.ppre, a.amin, a.was_ghost, a.gsum, a.gnu};
        for (void* b : bufs) free_one(c, b);
        a = AdjBuffers{};
        return rc;
    }
    a.ready = true;
    return MPS_OK;
}

}  // namespace
}  // namespace mps

using namespace mps;

struct mps_ctx : public mps::Ctx {};

extern "C" {

void mps_params_default(mps_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->dim = 2;
    p->pressure_mode = 0;
    p->l0 = 0.01;
    p->re_n = 2.1 * 0.01;
    p->re_lap = 4.0 * 0.01;
    p->rho = 1000.0;
    p->nu = 1e-6;
    p->dt = 1e-4;
    p->beta = 0.97;
    p->g[1] = -9.81;
    p->c0 = 20.0;
    p->gamma = 7.0;
    p->alpha_c = 1e-7;
    p->cg_tol = 1e-8;
    p->clamp_negative_p = 1;
    p->cell_skin = 0.1;
    p->box_max[0] = p->box_max[1] = p->box_max[2] = 1.0;
    p->inner_tol = 1e-4;
    p->max_outer = 30;
    p->step_graph = 1;
}

int mps_create(const double* pos, const double* vel, const int8_t* types, int64_t n,
               const mps_params* params, mps_ctx** out) {
    if (!out || !pos || !types || n <= 0 || n >= ((int64_t)1 << 31)) return MPS_EINVAL;
    int rc = check_params(params);
    if (rc) return rc;
    if ((rc = check_host_state(n, params->dim, pos, vel, types))) return rc;
    DeviceGuard dg(params->device);
    if (!dg.ok) return MPS_EDEVICE;
    mps_ctx* c = new (std::nothrow) mps_ctx();
    if (!c) return MPS_ENOMEM;
    c->prm = *params;
    c->n = n;
    c->steps_done = 0;
    c->cg_fused = params->inner_cg == 1;
    c->spmv_block = params->spmv_block ? params->spmv_block : 512;
    c->build_block = params->build_block;
    c->cg_unroll = params->cg_unroll ? params->cg_unroll : 1;
    c->predict_tpr = params->predict_tpr ? params->predict_tpr : 1;
    c->last_cg_iters = 8;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, params->device) != cudaSuccess) {
        delete c;
        return MPS_EDEVICE;
    }
    if (params->stream) {
        c->stream = (cudaStream_t)params->stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return MPS_EDEVICE;
        }
        c->own_stream = true;
    }
    if ((rc = setup(c, nullptr, 1)) || (rc = allocate(c)) || (rc = build_rows_init(c)) ||
        (rc = upload_state(c, pos, vel, types, false))) {
        mps_destroy(c);
        return rc;
    }
    *out = c;
    return MPS_OK;
}

int mps_create_ensemble(const double* pos, const double* vel, const int8_t* types,
                        const int32_t* scene, int64_t n, const mps_params* params,
                        const mps_scene* scenes, int32_t n_scenes, mps_ctx** out) {
    if (!out || !pos || !types || !scene || !scenes || n <= 0 || n >= ((int64_t)1 << 31) ||
        n_scenes < 1 || n_scenes > 65535)
        return MPS_EINVAL;
    if (!params) return MPS_EINVAL;
    mps_params P = *params;
    // the common parameters are checked with the first scene's box and spacing
    P.l0 = params->l0;
    for (int a = 0; a < 3; a++) {
        P.box_min[a] = scenes[0].box_min[a];
        P.box_max[a] = scenes[0].box_max[a];
    }
    int rc = check_params(&P);
    if (rc) return rc;
    if ((rc = check_host_state(n, P.dim, pos, vel, types))) return rc;
    std::vector<uint16_t> sid((size_t)n);
    for (int64_t i = 0; i < n; i++) {
        if (scene[i] < 0 || scene[i] >= n_scenes) return MPS_EINVAL;
        sid[(size_t)i] = (uint16_t)scene[i];
    }
    DeviceGuard dg(P.device);
    if (!dg.ok) return MPS_EDEVICE;
    mps_ctx* c = new (std::nothrow) mps_ctx();
    if (!c) return MPS_ENOMEM;
    c->prm = P;
    c->cg_fused = P.inner_cg == 1;
    c->spmv_block = P.spmv_block ? P.spmv_block : 512;
    c->build_block = P.build_block;
    c->cg_unroll = P.cg_unroll ? P.cg_unroll : 1;
    c->predict_tpr = P.predict_tpr ? P.predict_tpr : 1;
    c->scenes_host.assign(scenes, scenes + n_scenes);
    c->n = n;
    c->steps_done = 0;
    c->last_cg_iters = 8;
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess) {
        delete c;
        return MPS_EDEVICE;
    }
    if (P.stream) {
        c->stream = (cudaStream_t)P.stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return MPS_EDEVICE;
        }
        c->own_stream = true;
    }
    if ((rc = setup(c, scenes, n_scenes)) || (rc = allocate(c)) || (rc = build_rows_init(c))) {
        mps_destroy(c);
        return rc;
    }
    if (c->sid_id) {
        if (cudaMemcpyAsync(c->sid_id, sid.data(), sizeof(uint16_t) * sid.size(),
                            cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            mps_destroy(c);
            return MPS_EDEVICE;
        }
    }
    if ((rc = upload_state(c, pos, vel, types, false))) {
        mps_destroy(c);
        return rc;
    }
    *out = c;
    return MPS_OK;
}

int mps_autotune(mps_ctx* c, int32_t repeats, mps_tuning* out) {
    if (!c || repeats < 1) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    int rc;
    mps_tuning t;
    std::memset(&t, 0, sizeof t);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return MPS_EDEVICE;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return MPS_EDEVICE;
    }
    // mean time of `repeats` runs of f after one untimed run
    auto time_of = [&](auto&& f, float* ms) -> int {
        float total = 0.f;
        for (int r = 0; r <= repeats; r++) {
            cudaEventRecord(e0, c->stream);
            int frc = f();
            cudaEventRecord(e1, c->stream);
            if (frc) return frc;
            if (cudaEventSynchronize(e1) != cudaSuccess) return MPS_EDEVICE;
            float m = 0.f;
            cudaEventElapsedTime(&m, e0, e1);
            if (r > 0) total += m;
        }
        *ms = total / repeats;
        return MPS_OK;
    };
    const size_t n = (size_t)c->n;
    // ---- the cell side (after a step: the list skin then reflects the motion), timed as a
    // bucket build plus a candidate gather at the list skin of the next step
    t.cell_skin = c->prm.cell_skin;
    rc = [&]() -> int {
        if (c->steps_done < 1) return MPS_OK;
        const double s0 = c->prm.cell_skin;
        const double lo = std::max(0.05, 2.0 * c->list_skin);
        std::vector<double> cand{s0};
        for (double s : {0.05, 0.1, 0.15, 0.2})
            if (s >= lo && std::fabs(s - s0) > 1e-12) cand.push_back(s);
        if (cand.size() < 2) return MPS_OK;
        double best = s0;
        float best_ms = 1e30f;
        int r2;
        for (double s : cand) {
            r2 = regrid(c, s);
            if (r2 == MPS_ENOMEM) continue;   // the tables of a finer grid do not fit
            if (r2) return r2;
            if ((r2 = set_candidate_radius(c, c->list_skin))) return r2;
            auto run = [&]() -> int {
                MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
                int r3 = bucket_build(c, true);
                if (r3) return r3;
                MPS_CUDA(c, cudaMemsetAsync(c->vl_cnt, 0, n * sizeof(int32_t), c->stream));
                launch_verlet(c);
                return MPS_OK;
            };
            // both buffer parities' bucket graphs captured before the timed runs
            if ((r2 = run()) || (r2 = run())) return r2;
            float ms = 0.f;
            if ((r2 = time_of(run, &ms))) return r2;
            if (ms < best_ms) {
                best_ms = ms;
                best = s;
            }
        }
        if ((r2 = regrid(c, best))) return r2;
        t.cell_skin = best;
        t.cell_ms = best_ms;
        return MPS_OK;
    }();
    // ---- the candidate gather's block shape, on the current state
    if (!rc) rc = [&]() -> int {
        MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
        int r2 = bucket_build(c, true);
        if (r2) return r2;
        c->need_list = true;
        if ((r2 = set_candidate_radius(c, c->list_skin))) return r2;
        const int shapes[4] = {32, 64, 96, 128};
        int best = c->prm.gather_block;
        float best_ms = 1e30f;
        for (int b : shapes) {
            c->prm.gather_block = b;
            float ms = 0.f;
            r2 = time_of([&]() -> int {
                MPS_CUDA(c, cudaMemsetAsync(c->vl_cnt, 0, n * sizeof(int32_t), c->stream));
                launch_verlet(c);
                return MPS_OK;
            }, &ms);
            if (r2) return r2;
            if (ms < best_ms) {
                best_ms = ms;
                best = b;
            }
        }
        c->prm.gather_block = best;
        t.gather_block = best;
        t.gather_ms = best_ms;
        return MPS_OK;
    }();
    // ---- the prediction's threads per row and the row build's block, on the lists just
    // gathered (and the prediction from them)
    if (!rc) rc = [&]() -> int {
        MPS_CUDA(c, cudaMemsetAsync(c->vl_cnt, 0, n * sizeof(int32_t), c->stream));
        launch_verlet(c);
        launch_copy_state_star(c);
        {
            int best = c->predict_tpr, r2;
            float best_ms = 1e30f;
            for (int tpr : {1, 2, 4}) {
                c->predict_tpr = tpr;
                float ms = 0.f;
                r2 = time_of([&]() -> int {
                    launch_predict_rows(c);
                    return MPS_OK;
                }, &ms);
                if (r2) return r2;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = tpr;
                }
            }
            c->predict_tpr = best;
            t.predict_tpr = best;
            t.predict_ms = best_ms;
        }
        launch_predict_rows(c);
        if (c->prm.pressure_mode == 0 && c->prm.source_term == 2) launch_ecs_rates(c);
        int best = build_block_of(c), r2;
        float best_ms = 1e30f;
        for (int b : {64, 128, 256}) {
            c->build_block = b;
            float ms = 0.f;
            r2 = time_of([&]() -> int {
                launch_build_rows(c);
                return MPS_OK;
            }, &ms);
            if (r2) return r2;
            if (ms < best_ms) {
                best_ms = ms;
                best = b;
            }
        }
        c->build_block = best;
        t.build_block = best;
        t.build_ms = best_ms;
        return MPS_OK;
    }();
    // ---- the mixed PPE: the FP32 SpMV's block size and the inner CG's form, on the system
    // of a solve at the current state (the state is not advanced)
    const bool mixed_ppe = c->prm.pressure_mode == 0 && c->prm.precision == 1;
    if (!rc && mixed_ppe) {
        rc = [&]() -> int {
            mps_report rep;
            std::memset(&rep, 0, sizeof rep);
            int r2 = do_step(c, false, &rep);
            if (r2 && r2 != MPS_ECG_NOCONV) return r2;
            float best_ms = 1e30f;
            int best = c->spmv_block;
            for (int b : {256, 512}) {
                c->spmv_block = b;
                double ms = 0.0, bytes = 0.0;
                if ((r2 = ppe_time_kernel(c, 0, repeats, &ms, &bytes))) return r2;
                if (ms < best_ms) {
                    best_ms = (float)ms;
                    best = b;
                }
            }
            c->spmv_block = best;
            t.spmv_block = best;
            t.spmv_ms = best_ms;
            if (c->prm.ppe_host_loop != 0) return MPS_OK;   // the fused form is device-driven only
            best_ms = 1e30f;
            bool best_f = c->cg_fused;
            int best_u = c->cg_unroll;
            for (bool f : {false, true}) {
                for (int u : {1, 2, 4}) {
                    c->cg_fused = f;
                    c->cg_unroll = u;
                    ppe_graphs_destroy(c);
                    float ms = 0.f;
                    r2 = time_of([&]() -> int {
                        mps_report pr;
                        std::memset(&pr, 0, sizeof pr);
                        int r3 = ppe_solve(c, &pr);
                        return (r3 == MPS_ECG_NOCONV) ? MPS_OK : r3;
                    }, &ms);
                    if (r2) return r2;
                    if (ms < best_ms) {
                        best_ms = ms;
                        best_f = f;
                        best_u = u;
                    }
                }
            }
            c->cg_fused = best_f;
            c->cg_unroll = best_u;
            ppe_graphs_destroy(c);
            t.cg_fused = best_f ? 1 : 0;
            t.cg_unroll = best_u;
            t.solve_ms = best_ms;
            return MPS_OK;
        }();
    } else {
        t.spmv_block = c->spmv_block;
        t.cg_fused = c->cg_fused ? 1 : 0;
        t.cg_unroll = c->cg_unroll;
        if (!rc) {
            // p, n* and flags of a solve at the current state, as after the mixed PPE's tuning
            mps_report rep;
            std::memset(&rep, 0, sizeof rep);
            rc = do_step(c, false, &rep);
            if (rc == MPS_ECG_NOCONV) rc = MPS_OK;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    step_graphs_destroy(c);   // they captured the tuned kernels' launch shapes
    if (rc) return rc;
    MPS_CUDA(c, cudaGetLastError());
    if (out) *out = t;
    return MPS_OK;
}

int mps_scene_residuals(mps_ctx* c, double* out) {
    if (!c || !out) return MPS_EINVAL;
    for (int s = 0; s < c->n_scenes; s++) out[s] = c->scene_resid[(size_t)s];
    return MPS_OK;
}

int mps_step(mps_ctx* c, int32_t nsteps, mps_report* last) {
    if (!c || nsteps < 0) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    mps_report rep;
    std::memset(&rep, 0, sizeof rep);
    rep.steps_done = c->steps_done;
    int rc = MPS_OK;
    for (int k = 0; k < nsteps && rc == MPS_OK; k++) rc = do_step(c, true, &rep);
    rep.status = rc;
    if (last) *last = rep;
    return rc;
}

int mps_solve_ppe(mps_ctx* c, mps_report* out) {
    if (!c) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    mps_report rep;
    std::memset(&rep, 0, sizeof rep);
    int rc = do_step(c, false, &rep);
    rep.status = rc;
    if (out) *out = rep;
    return rc;
}

int mps_clear_history(mps_ctx* c) {
    if (!c) return MPS_EINVAL;
    c->guess_n = 0;
    return MPS_OK;
}

int mps_set_gravity(mps_ctx* c, const double* g) {
    if (!c || !g) return MPS_EINVAL;
    for (int a = 0; a < 3; a++)
        if (!std::isfinite(g[a])) return MPS_EINVAL;
    for (int a = 0; a < 3; a++) c->prm.g[a] = g[a];
    return MPS_OK;
}


namespace {
int step_vjp(Ctx* c, const double* g_pos, const double* g_vel, double* out_pos, double* out_vel,
             double* out_g, double* out_nu, mps_vjp_report* out, bool device) {
    if (!c || !g_pos || !g_vel || !out_pos || !out_vel) return MPS_EINVAL;
    const cudaMemcpyKind in = device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind back = device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const mps_params& P = c->prm;
    if (c->n_scenes > 1 || P.kernel != 0 || P.gradient_form != 0 || P.source_term != 0)
        return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    mps_vjp_report vr;
    std::memset(&vr, 0, sizeof vr);
    int rc = alloc_adjoint(c);
    if (rc) return rc;
    const size_t n = (size_t)c->n, dim = (size_t)c->dim;
    // the forward step from the current state, kept for the reverse: fresh candidate lists
    // (DUMMY rows included), the PPE solution before the clamp
    launch_adj_mark(c);
    c->vjp = true;
    c->need_list = true;
    rc = do_step(c, false, &vr.forward);
    c->vjp = false;
    c->need_list = true;   // the next step gathers its own lists (without DUMMY rows)
    vr.forward.status = rc;
    if (rc) {
        vr.status = rc;
        if (out) *out = vr;
        return rc;
    }
    double* d_a = (double*)c->stage;
    double* d_b = d_a + n * dim;
    MPS_CUDA(c, cudaMemcpyAsync(d_a, g_pos, n * dim * sizeof(double), in, c->stream));
    MPS_CUDA(c, cudaMemcpyAsync(d_b, g_vel, n * dim * sizeof(double), in, c->stream));
    launch_adj_load(c, d_a, d_b);
    launch_adj_front(c);
    if (P.pressure_mode == 0) {
        mps_report ar;
        std::memset(&ar, 0, sizeof ar);
        rc = ppe_solve_rhs(c, c->adj.lam, c->adj.pbar, &ar);
        vr.cg_iters = ar.cg_iters;
        vr.cg_outer = ar.cg_outer;
        vr.cg_resid = ar.cg_resid;
        if (rc) {
            vr.status = rc;
            if (out) *out = vr;
            return rc;
        }
    }
    launch_adj_back(c, c->adj.gsum);
    double* d_nu = out_nu ? (device ? out_nu : d_b + n * dim) : nullptr;
    launch_adj_store(c, d_a, d_b, d_nu);
    MPS_CUDA(c, cudaGetLastError());
    MPS_CUDA(c, cudaMemcpyAsync(out_pos, d_a, n * dim * sizeof(double), back, c->stream));
    MPS_CUDA(c, cudaMemcpyAsync(out_vel, d_b, n * dim * sizeof(double), back, c->stream));
    if (out_nu && !device)
        MPS_CUDA(c, cudaMemcpyAsync(out_nu, d_nu, n * sizeof(double), cudaMemcpyDeviceToHost,
                                    c->stream));
    double gs[3] = {0.0, 0.0, 0.0};
    MPS_CUDA(c, cudaMemcpyAsync(gs, c->adj.gsum, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    if (out_g)
        for (int a = 0; a < 3; a++) out_g[a] = a < c->dim ? gs[a] : 0.0;
    if (out) *out = vr;
    return MPS_OK;
}
}  // namespace

int mps_step_vjp(mps_ctx* c, const double* g_pos, const double* g_vel, double* out_pos,
                 double* out_vel, double* out_g, double* out_nu, mps_vjp_report* out) {
    return step_vjp(c, g_pos, g_vel, out_pos, out_vel, out_g, out_nu, out, false);
}

int mps_step_vjp_device(mps_ctx* c, const double* g_pos, const double* g_vel, double* out_pos,
                        double* out_vel, double* out_g, double* out_nu, mps_vjp_report* out) {
    return step_vjp(c, g_pos, g_vel, out_pos, out_vel, out_g, out_nu, out, true);
}

namespace {
int read_state(Ctx* c, double* pos, double* vel, double* p, double* n_star, uint8_t* flags,
               int8_t* types, cudaMemcpyKind out) {
    if (!c) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    const size_t n = (size_t)c->n, dim = (size_t)c->dim;
    uint8_t* base = (uint8_t*)c->stage;
    double* d_pos = (double*)base;
    double* d_vel = d_pos + n * dim;
    double* d_p = d_vel + n * dim;
    double* d_n = d_p + n;
    uint8_t* d_f = (uint8_t*)(d_n + n);
    int8_t* d_t = (int8_t*)(d_f + n);
    launch_unpermute(c, pos ? d_pos : nullptr, vel ? d_vel : nullptr, p ? d_p : nullptr,
                     n_star ? d_n : nullptr, flags ? d_f : nullptr, types ? d_t : nullptr);
    MPS_CUDA(c, cudaGetLastError());
    if (pos) MPS_CUDA(c, cudaMemcpyAsync(pos, d_pos, n * dim * 8, out, c->stream));
    if (vel) MPS_CUDA(c, cudaMemcpyAsync(vel, d_vel, n * dim * 8, out, c->stream));
    if (p) MPS_CUDA(c, cudaMemcpyAsync(p, d_p, n * 8, out, c->stream));
    if (n_star) MPS_CUDA(c, cudaMemcpyAsync(n_star, d_n, n * 8, out, c->stream));
    if (flags) MPS_CUDA(c, cudaMemcpyAsync(flags, d_f, n, out, c->stream));
    if (types) MPS_CUDA(c, cudaMemcpyAsync(types, d_t, n, out, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    return MPS_OK;
}
}  // namespace

int mps_read_state(mps_ctx* c, double* pos, double* vel, double* p, double* n_star,
                   uint8_t* flags, int8_t* types) {
    return read_state(c, pos, vel, p, n_star, flags, types, cudaMemcpyDeviceToHost);
}

int mps_read_state_device(mps_ctx* c, double* pos, double* vel, double* p, double* n_star,
                          uint8_t* flags, int8_t* types) {
    return read_state(c, pos, vel, p, n_star, flags, types, cudaMemcpyDeviceToDevice);
}

int mps_write_state(mps_ctx* c, const double* pos, const double* vel, const int8_t* types) {
    if (!c || !pos) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    // the same checks as mps_create, on the device (a restart path uploads every step)
    return upload_state(c, pos, vel, types, true, true);
}

int mps_write_state_device(mps_ctx* c, const double* pos, const double* vel, const int8_t* types) {
    if (!c || !pos) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    return upload_state(c, pos, vel, types, true, true, true);
}

int mps_set_fluid_properties(mps_ctx* c, const double* rho, const double* nu) {
    if (!c) return MPS_EINVAL;
    const int64_t n = c->n;
    if (rho) {
        if (c->prm.pressure_mode == 0 && c->prm.ppe_operator == 1) return MPS_EINVAL;
        for (int64_t i = 0; i < n; i++)
            if (!(std::isfinite(rho[i]) && rho[i] > 0.0)) return MPS_EINVAL;
    }
    if (nu)
        for (int64_t i = 0; i < n; i++)
            if (!(std::isfinite(nu[i]) && nu[i] >= 0.0)) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    const size_t bytes = (size_t)n * sizeof(double);
    int rc;
    // the buffers are taken all or none: a context never sees half of a property's set
    if (rho) {
        if (!c->rho_id) {
            double *a = nullptr, *b = nullptr;
            float2* f = nullptr;
            if ((rc = alloc_dev(c, &a, (size_t)n)) || (rc = alloc_dev(c, &b, (size_t)n)) ||
                (rc = alloc_dev(c, &f, (size_t)n))) {
                free_one(c, a);
                free_one(c, b);
                free_one(c, f);
                return rc;
            }
            c->rho_id = a;
            c->rho_s = b;
            c->rho_ff = f;
        }
        MPS_CUDA(c, cudaMemcpyAsync(c->rho_id, rho, bytes, cudaMemcpyHostToDevice, c->stream));
    } else if (c->rho_id) {
        free_one(c, c->rho_id);
        free_one(c, c->rho_s);
        free_one(c, c->rho_ff);
        c->rho_id = c->rho_s = nullptr;
        c->rho_ff = nullptr;
    }
    if (nu) {
        if (!c->nu_id) {
            double *a = nullptr, *b = nullptr;
            if ((rc = alloc_dev(c, &a, (size_t)n)) || (rc = alloc_dev(c, &b, (size_t)n))) {
                free_one(c, a);
                free_one(c, b);
                return rc;
            }
            c->nu_id = a;
            c->nu_s = b;
        }
        MPS_CUDA(c, cudaMemcpyAsync(c->nu_id, nu, bytes, cudaMemcpyHostToDevice, c->stream));
    } else if (c->nu_id) {
        free_one(c, c->nu_id);
        free_one(c, c->nu_s);
        c->nu_id = c->nu_s = nullptr;
    }
    launch_gather_props(c);
    MPS_CUDA(c, cudaGetLastError());
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    bucket_graphs_destroy(c);   // the captured builds gather the properties that were set
    step_graphs_destroy(c);
    return MPS_OK;
}

int mps_debug_cells(mps_ctx* c, uint32_t* cell_key) {
    if (!c || !cell_key || c->n_scenes > 1) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    uint32_t* d_out = (uint32_t*)c->stage;
    launch_cell_keys_only(c, c->key_alt);
    launch_unpermute_u32(c, c->key_alt, d_out);
    MPS_CUDA(c, cudaGetLastError());
    MPS_CUDA(c, cudaMemcpyAsync(cell_key, d_out, (size_t)c->n * 4, cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    return MPS_OK;
}

int mps_debug_neighbors(mps_ctx* c, int32_t which, int64_t* offsets, int32_t* ids, int64_t cap) {
    if (!c || !offsets || (which != 0 && which != 1) || c->n_scenes > 1) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    const int n = (int)c->n;
    int rc;
    MPS_CUDA(c, cudaMemsetAsync(c->st, 0, sizeof(DevStatus), c->stream));
    if ((rc = bucket_build(c, false))) return rc;
    c->need_list = true;   // the state was reordered: kept candidate lists no longer apply
    const Radius& r = which == 0 ? c->r_n : c->r_lap;
    int32_t* d_cnt = nullptr;
    int64_t* d_off = nullptr;
    int32_t* d_ids = nullptr;
    if ((rc = alloc_dev(c, &d_cnt, (size_t)n))) return rc;
    MPS_CUDA(c, cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * n, c->stream));
    launch_debug_neighbors(c, r, nullptr, nullptr, d_cnt);
    std::vector<int32_t> cnt(n), slot_id(n);
    MPS_CUDA(c, cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaMemcpyAsync(slot_id.data(), c->id, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<int64_t> soff(n + 1, 0);
    for (int s = 0; s < n; s++) soff[s + 1] = soff[s] + cnt[s];
    // offsets in original order
    std::vector<int64_t> ocnt(n, 0);
    for (int s = 0; s < n; s++) ocnt[slot_id[s]] = cnt[s];
    offsets[0] = 0;
    for (int i = 0; i < n; i++) offsets[i + 1] = offsets[i] + ocnt[i];
    const int64_t total = soff[n];
    if (!ids) {
        free_one(c, d_cnt);
        return MPS_OK;
    }
    if (total > cap) {
        free_one(c, d_cnt);
        return MPS_ECAP;
    }
    if ((rc = alloc_dev(c, &d_off, (size_t)n + 1)) || (rc = alloc_dev(c, &d_ids, (size_t)std::max<int64_t>(total, 1)))) {
        free_one(c, d_cnt);
        if (d_off) free_one(c, d_off);
        return rc;
    }
    MPS_CUDA(c, cudaMemcpyAsync(d_off, soff.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    launch_debug_neighbors(c, r, d_off, d_ids, d_cnt);
    std::vector<int32_t> sids(std::max<int64_t>(total, 1));
    MPS_CUDA(c, cudaMemcpyAsync(sids.data(), d_ids, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int s = 0; s < n; s++) {
        const int i = slot_id[s];
        int32_t* dst = ids + offsets[i];
        std::copy(sids.begin() + soff[s], sids.begin() + soff[s + 1], dst);
        std::sort(dst, dst + cnt[s]);
    }
    free_one(c, d_cnt);
    free_one(c, d_off);
    free_one(c, d_ids);
    return MPS_OK;
}

int mps_get_constants(mps_ctx* c, double* out) {
    if (!c || !out) return MPS_EINVAL;
    out[0] = c->n0_pnd;
    out[1] = c->n0_lap;
    out[2] = c->lambda;
    out[3] = c->h;
    out[4] = c->grid.ncell[0];
    out[5] = c->grid.ncell[1];
    out[6] = c->grid.ncell[2];
    out[7] = c->cap;
    return MPS_OK;
}

int mps_set_profiling(mps_ctx* c, int32_t on) {
    if (!c) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    if (on && !c->ev[0]) {
        for (int k = 0; k < 2 * MPS_NSTAGES; k++)
            MPS_CUDA(c, cudaEventCreate(&c->ev[k]));
    }
    c->profiling = on != 0;
    c->launches = 0;
    for (int s = 0; s < MPS_NSTAGES; s++) {
        c->stage_ms[s] = 0.0;
        c->stage_calls[s] = 0;
    }
    return MPS_OK;
}

int mps_time_kernel(mps_ctx* c, int32_t which, int32_t repeats, double* ms_per_launch,
                    double* bytes_per_launch) {
    if (!c || !ms_per_launch || !bytes_per_launch) return MPS_EINVAL;
    DeviceGuard dg(c->prm.device);
    if (!dg.ok) return MPS_EDEVICE;
    return ppe_time_kernel(c, which, repeats, ms_per_launch, bytes_per_launch);
}

int mps_get_profile(mps_ctx* c, double* stage_ms, int64_t* stage_calls, int64_t* launches) {
    if (!c) return MPS_EINVAL;
    for (int s = 0; s < MPS_NSTAGES; s++) {
        if (stage_ms) stage_ms[s] = c->stage_ms[s];
        if (stage_calls) stage_calls[s] = c->stage_calls[s];
    }
    if (launches) *launches = c->launches;
    return MPS_OK;
}

void mps_destroy(mps_ctx* c) {
    if (!c) return;
    {
        DeviceGuard dg(c->prm.device);
        if (c->stream) cudaStreamSynchronize(c->stream);
        for (int k = 0; k < 2 * MPS_NSTAGES; k++)
            if (c->ev[k]) cudaEventDestroy(c->ev[k]);
        ppe_graphs_destroy(c);
        bucket_graphs_destroy(c);
        step_graphs_destroy(c);
        if (c->ctl_host) cudaFreeHost(c->ctl_host);
        if (c->rv_var_host) cudaFreeHost(c->rv_var_host);
        if (c->scene_sums_host) cudaFreeHost(c->scene_sums_host);
        free_all(c);
        if (c->st_host) cudaFreeHost(c->st_host);
        if (c->cg_host) cudaFreeHost(c->cg_host);
        if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    }
    delete c;
}

const char* mps_strerror(int status) {
    switch (status) {
        case MPS_OK: return "MPS_OK";
        case MPS_EINVAL: return "MPS_EINVAL: invalid argument";
        case MPS_ENOMEM: return "MPS_ENOMEM: allocation failed";
        case MPS_ECG_NOCONV: return "MPS_ECG_NOCONV: CG did not converge within cg_max_iter";
        case MPS_ENONFINITE: return "MPS_ENONFINITE: non-finite position or velocity";
        case MPS_ESKIN: return "MPS_ESKIN: a particle moved more than half the cell skin";
        case MPS_ECOINCIDENT: return "MPS_ECOINCIDENT: two neighbouring particles coincide";
        case MPS_ECAP: return "MPS_ECAP: neighbour capacity exceeded";
        case MPS_EDEVICE: return "MPS_EDEVICE: CUDA error";
        default: return "unknown status";
    }
}

}  // extern "C"
