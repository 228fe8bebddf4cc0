// update.cu -- pressure clamp and minimum pressure, gradient correction, state transfers.
//
// Clamp / p_hat (PPE path): p_i = max(p_i, 0); p_hat_i = min(p_i, min_j p_j) over the
// non-dummy neighbours j within re_n at r* (the stabilising p_hat of the gradient).
// Gradient (difference form of the multi-density gradient of Sec. 3.2.1, one density):
//   grad p_i = d/n0 sum_j (p_j - p_hat_i)/|r_ij|^2 r_ij w(|r_ij|),  r_ij = r*_j - r*_i,
// over non-dummy j within re_n; FLUID only:
//   u' = -(dt/rho) grad p_i,  u = u* + u',  r = r* + dt u'   (first-order Euler, Sec. 3.1).
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 256;

__global__ void __launch_bounds__(kBT)
    k_clamp_pmin(int n, const int8_t* type, double* p, double* phat, const int32_t* ncol,
                 const int32_t* ncnt, int cap_n, int clamp, int walls) {
    int i = blockIdx.x * kBT + threadIdx.x;
    if (i >= n) return;
    double pi = p[i];
    if (clamp) pi = fmax(pi, 0.0);
    double m = pi;
    if (type[i] == kFluid || (walls && type[i] == kWall)) {   // wall p_hat: CMPS pair terms
        const int cnt = ncnt[i];
        for (int k = 0; k < cnt; k++) {
            double pj = p[ncol[sell8(i, k, cap_n)]];
            if (clamp) pj = fmax(pj, 0.0);
            m = fmin(m, pj);
        }
    }
    phat[i] = m;
}

// the guess history of the PPE: h_2 <- h_1, h_1 <- h_0, h_0 <- p (as many as are kept)
__global__ void __launch_bounds__(kBT) k_push_history(int n, int m, double* h0, double* h1,
                                                      double* h2, double* h3, const double* p) {
    const int i = blockIdx.x * kBT + threadIdx.x;
    if (i >= n) return;
    if (m >= 4) h3[i] = h2[i];
    if (m >= 3) h2[i] = h1[i];
    if (m >= 2) h1[i] = h0[i];
    h0[i] = p[i];
}

// p was clamped on read above; store the clamped values once every p_hat is computed
__global__ void __launch_bounds__(kBT) k_clamp_store(int n, double* p) {
    int i = blockIdx.x * kBT + threadIdx.x;
    if (i < n) p[i] = fmax(p[i], 0.0);
}

// Per-row extras of the update: the two-phase density, and for candidate lists kept across
// steps the refresh of the FP32 copies of r, u and r^{k+1} measured against the positions
// r_b the lists were gathered at.
struct Keep {
    int kernel;             // 0: re/r - 1 (Eq. 4); 1: (1 - r/re)^3
    int form;               // 0: (p_j - p_hat_i); 1: CMPS (Eq. 18)
    int phat_mode;          // p_hat_i: 0 read from phat; 1 min(p_i, min_j p_j) over the row's
                            // list, taken here; 2 p_i (the equation of state)
    double inv_re;          // 1/re_n
    float inv_f;
    const double* rho_s;    // two-phase: per-slot density (null: the uniform rho)
    const uint16_t* sid;    // ensemble: scene of every slot (null: one scene)
    const SceneParams* scn;
    const double4* pos_b;   // null: lists are gathered every step (nothing else is used)
    float4* pos32;
    float4* pos32lo;
    float4* vel32;
    GridDesc g;
    DevStatus* st;
};

// One FLUID row of the pressure-gradient correction; returns |r^{k+1} - r_b|^2 when
// candidate lists are kept (0 otherwise)
template <bool MIXED>
__device__ __forceinline__ double gradient_row(int i, const int8_t* type, const double4* ps,
                                               const float4* ps32, const double4* us,
                                               const double* p, const double* phat,
                                               const int32_t* ncol, const int32_t* ncnt, int cap_n,
                                               double re, float re_f, double coef_grad, double dt,
                                               double rho, double4* pos, double4* vel,
                                               const Keep& kp) {
    const double4 pi = ps[i];
    const double pp = p[i];
    const int cnt = ncnt[i];
    double ph = kp.phat_mode == 2 ? pp : (kp.phat_mode == 1 ? pp : phat[i]);
    if (kp.phat_mode == 1) {
        // the neighbourhood minimum (p already clamped in memory when the clamp is on): the
        // same values and the same exact min as a separate pass
        for (int k = 0; k < cnt; k++) ph = fmin(ph, p[ncol[sell8(i, k, cap_n)]]);
    }
    double inv_re = kp.inv_re;
    float inv_f = kp.inv_f;
    if (kp.sid) {   // ensemble: the row's scene
        const SceneParams& sp = kp.scn[kp.sid[i]];
        re = sp.rn.re;
        re_f = sp.rn.re_f;
        coef_grad = sp.coef_grad;
        inv_re = sp.rn.inv_re;
        inv_f = sp.rn.inv_f;
    }
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (MIXED) {
        const float4 qi = ps32[i];
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        for (int k = 0; k < cnt; k++) {
            const int j = ncol[sell8(i, k, cap_n)];
            const float4 qj = ps32[j];
            const float dx = qj.x - qi.x, dy = qj.y - qi.y, dz = qj.z - qi.z;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rs = rsqrtf(r2);
            const float w = kp.kernel == 1 ? cubic_w_f(r2, rs, inv_f) : fmaf(re_f, rs, -1.f);
            const double dp = kp.form == 1 ? (pp + p[j]) - (ph + phat[j]) : p[j] - ph;
            const float f = (float)dp * (w * rs * rs);
            f0 = fmaf(f, dx, f0);
            f1 = fmaf(f, dy, f1);
            f2 = fmaf(f, dz, f2);
        }
        g0 = f0;
        g1 = f1;
        g2 = f2;
    } else {
        for (int k = 0; k < cnt; k++) {
            const int j = ncol[sell8(i, k, cap_n)];
            const double4 pj = ps[j];
            const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const double r2 = fma(dz, dz, fma(dy, dy, dx * dx));
            const double rs = rsqrt(r2);
            const double w = kp.kernel == 1 ? cubic_w_d(r2, rs, inv_re) : fma(re, rs, -1.0);
            const double dp = kp.form == 1 ? (pp + p[j]) - (ph + phat[j]) : p[j] - ph;
            const double f = dp * (w * rs * rs);
            g0 = fma(f, dx, g0);
            g1 = fma(f, dy, g1);
            g2 = fma(f, dz, g2);
        }
    }
    const double k = -(dt / (kp.rho_s ? kp.rho_s[i] : rho)) * coef_grad;
    const double4 u = us[i];
    const double d0 = k * g0, d1 = k * g1, d2 = k * g2;
    const double4 un = make_double4(u.x + d0, u.y + d1, u.z + d2, 0.0);
    const double4 xn = make_double4(pi.x + dt * d0, pi.y + dt * d1, pi.z + dt * d2, 0.0);
    vel[i] = un;
    pos[i] = xn;
    if (kp.pos_b == nullptr) return 0.0;
    // the next step starts without a bucket build: refresh the FP32 copies at r^{k+1} and
    // flag a particle that leaves the cell grid (or is not finite) for a fresh gather
    const GridDesc& g = kp.g;
    float4 h4, l4;
    split_rel(xn.x, g.bmin[0], &h4.x, &l4.x);
    split_rel(xn.y, g.bmin[1], &h4.y, &l4.y);
    split_rel(xn.z, g.bmin[2], &h4.z, &l4.z);
    h4.w = __int_as_float((int)type[i]);
    l4.w = 0.f;
    kp.pos32[i] = h4;
    kp.pos32lo[i] = l4;
    kp.vel32[i] = make_float4((float)un.x, (float)un.y, (float)un.z, 0.f);
    const double xs[3] = {xn.x, xn.y, xn.z};
    bool inside = isfinite(un.x) && isfinite(un.y) && isfinite(un.z);
    for (int a = 0; a < g.dim; a++) {
        const double q = cell_floor(__dsub_rn(xs[a], g.bmin[a]), g.h, g.inv_h, g.inv_hf);
        if (!(q >= 0.0 && q < (double)g.ncell[a])) inside = false;
    }
    if (!inside) atomicAdd(&kp.st->leave, 1u);
    const double4 b = kp.pos_b[i];
    const double ex = xn.x - b.x, ey = xn.y - b.y, ez = xn.z - b.z;
    return fma(ez, ez, fma(ey, ey, ex * ex));
}

template <bool MIXED>
__global__ void __launch_bounds__(kBT)
    k_gradient(int n, const int8_t* type, const double4* ps, const float4* ps32, const double4* us,
               const double* p, const double* phat, const int32_t* ncol, const int32_t* ncnt,
               int cap_n, double re, float re_f, double coef_grad, double dt, double rho,
               double4* pos, double4* vel, const int32_t* rows, const uint32_t* nrows, Keep kp) {
    // one thread per FLUID row (the bucket build's list of FLUID slots)
    const int tid = blockIdx.x * kBT + threadIdx.x;
    const int i = tid < (int)*nrows ? rows[tid] : -1;
    const bool act = i >= 0;
    if (kp.pos_b == nullptr && !act) return;
    double disp = 0.0;
    if (act) disp = gradient_row<MIXED>(i, type, ps, ps32, us, p, phat, ncol, ncnt, cap_n, re, re_f,
                                        coef_grad, dt, rho, pos, vel, kp);
    if (kp.pos_b == nullptr) return;
    // kept candidate lists: the largest |r^{k+1} - r_b| of the warp
    unsigned long long v = (unsigned long long)__double_as_longlong(disp);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v) atomicMax(&kp.st->max_disp_next_bits, v);
}

__global__ void __launch_bounds__(kBT)
    k_unpermute(int n, int dim, const int32_t* id, const double4* pos, const double4* vel,
                const double* p, const double* nstar, const uint8_t* flag, const int8_t* type,
                double* o_pos, double* o_vel, double* o_p, double* o_n, uint8_t* o_f, int8_t* o_t) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n) return;
    const int i = id[s];
    const double4 x = pos[s], u = vel[s];
    const double xa[3] = {x.x, x.y, x.z}, ua[3] = {u.x, u.y, u.z};
    for (int a = 0; a < dim; a++) {
        if (o_pos) o_pos[(size_t)i * dim + a] = xa[a];
        if (o_vel) o_vel[(size_t)i * dim + a] = ua[a];
    }
    if (o_p) o_p[i] = p[s];
    if (o_n) o_n[i] = nstar[s];
    if (o_f) o_f[i] = flag[s];
    if (o_t) o_t[i] = type[s];
}

__global__ void __launch_bounds__(kBT) k_unpermute_u32(int n, const int32_t* id, const uint32_t* in,
                                                       uint32_t* out) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s < n) out[id[s]] = in[s];
}

// a staged caller state before it replaces the context's: finite positions and velocities,
// known kinds (flags in the status word; nothing is written elsewhere)
__global__ void __launch_bounds__(kBT)
    k_check_stage(int n, int dim, const double* i_pos, const double* i_vel, const int8_t* i_t,
                  DevStatus* st) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n) return;
    bool fin = true;
    for (int a = 0; a < dim; a++) {
        fin = fin && isfinite(i_pos[(size_t)s * dim + a]);
        if (i_vel) fin = fin && isfinite(i_vel[(size_t)s * dim + a]);
    }
    if (!fin) atomicOr(&st->err, kErrNonfinite);
    if (i_t && (i_t[s] < kFluid || i_t[s] > kGhost)) atomicOr(&st->err, kErrKind);
}

// whether a staged caller state (original order) equals the context's, bit for bit: the
// positions, and the velocities and kinds where given
__global__ void __launch_bounds__(kBT)
    k_same_state(int n, int dim, const double* i_pos, const double* i_vel, const int8_t* i_t,
                 const double4* pos, const double4* vel, const int8_t* type, const int32_t* id,
                 DevStatus* st) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n) return;
    const size_t i = (size_t)id[s];
    const double4 x = pos[s], u = vel[s];
    const double xs[3] = {x.x, x.y, x.z}, us[3] = {u.x, u.y, u.z};
    bool same = !i_t || i_t[i] == type[s];
    for (int a = 0; a < dim; a++) {
        same = same && __double_as_longlong(i_pos[i * dim + a]) == __double_as_longlong(xs[a]);
        if (i_vel) same = same && __double_as_longlong(i_vel[i * dim + a]) == __double_as_longlong(us[a]);
    }
    if (!same) atomicOr(&st->differs, 1u);
}

// state from caller order; slot s = particle s (identity order until the next sort)
__global__ void __launch_bounds__(kBT)
    k_ingest(int n, int dim, const double* i_pos, const double* i_vel, const int8_t* i_t,
             double4* pos, double4* vel, int8_t* type, int32_t* id, double* p, double* nstar,
             uint8_t* flag, int keep_vel, int keep_types, GridDesc g, float4* pos32,
             float4* pos32lo) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n) return;
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < dim; a++) x[a] = i_pos[(size_t)s * dim + a];
    pos[s] = make_double4(x[0], x[1], x[2], 0.0);
    if (!keep_vel) {
        double u[3] = {0.0, 0.0, 0.0};
        if (i_vel)
            for (int a = 0; a < dim; a++) u[a] = i_vel[(size_t)s * dim + a];
        vel[s] = make_double4(u[0], u[1], u[2], 0.0);
    }
    if (!keep_types) type[s] = i_t[s];
    id[s] = s;
    p[s] = 0.0;
    nstar[s] = 0.0;
    flag[s] = 0;
    float4 h, l;
    split_rel(x[0], g.bmin[0], &h.x, &l.x);
    split_rel(x[1], g.bmin[1], &h.y, &l.y);
    split_rel(x[2], g.bmin[2], &h.z, &l.z);
    h.w = __int_as_float((int)type[s]);
    l.w = 0.f;
    pos32[s] = h;
    pos32lo[s] = l;
}
// per-particle properties into slot order (slot s holds particle id[s]): two-phase density
// (also as float-float for the pair factors of the mixed build) and viscosity, and the
// scene of an ensemble
__global__ void __launch_bounds__(kBT)
    k_gather_props(int n, const int32_t* id, const double* rho_id, const double* nu_id,
                   double* rho_s, double* nu_s, float2* rho_ff, const uint16_t* sid_id,
                   uint16_t* sid) {
    int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n) return;
    const int q = id[s];
    if (sid_id) sid[s] = sid_id[q];
    if (rho_id) {
        const double r = rho_id[q];
        const float h = (float)r;
        rho_s[s] = r;
        rho_ff[s] = make_float2(h, (float)(r - (double)h));
    }
    if (nu_id) nu_s[s] = nu_id[q];
}
}  // namespace

// With the difference-form gradient p_hat is needed by the gradient of FLUID rows only: the
// gradient kernel takes it from the row's own list (after the clamp is stored), which saves a
// pass over the lists; the reverse step, which keeps p_hat, and CMPS (p_hat_j of every
// neighbour) use the separate pass.
static bool phat_inline(const Ctx* c) { return c->prm.gradient_form == 0 && !c->vjp; }

void launch_push_history(Ctx* c) {
    const int n = (int)c->n;
    k_push_history<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->guess_m, c->ph[0], c->ph[1],
                                                               c->ph[2], c->ph[3], c->p);
    c->launches += 1;
}

int launch_pressure_floor(Ctx* c) {
    const int n = (int)c->n;
    const int nb = (n + kBT - 1) / kBT;
    const bool ppe = c->prm.pressure_mode == 0;
    if (phat_inline(c)) {
        if (ppe && c->prm.clamp_negative_p) {
            k_clamp_store<<<nb, kBT, 0, c->stream>>>(n, c->p);
            c->launches += 1;
        }
        return MPS_OK;
    }
    if (ppe || c->prm.gradient_form == 1) {
        launch_clamp_pmin(c);   // the equation of state clamps nothing (no PPE solve)
    } else {
        MPS_CUDA(c, cudaMemcpyAsync(c->phat, c->p, sizeof(double) * (size_t)n,
                                    cudaMemcpyDeviceToDevice, c->stream));
    }
    return MPS_OK;
}

void launch_clamp_pmin(Ctx* c) {
    const int n = (int)c->n;
    const int nb = (n + kBT - 1) / kBT;
    // the clamp belongs to the PPE solution; the equation of state's pressure is kept
    const int clamp = (c->prm.pressure_mode == 0 && c->prm.clamp_negative_p) ? 1 : 0;
    k_clamp_pmin<<<nb, kBT, 0, c->stream>>>(n, c->type, c->p, c->phat, c->nb_n_col, c->nb_n_cnt,
                                            c->cap_n, clamp, c->prm.gradient_form == 1 ? 1 : 0);
    if (clamp) k_clamp_store<<<nb, kBT, 0, c->stream>>>(n, c->p);
    c->launches += clamp ? 2 : 1;
}

void launch_gradient_correct(Ctx* c) {
    const int n = (int)c->n;
    const int nb = (n + kBT - 1) / kBT;
    const mps_params& P = c->prm;
    Keep kp;
    kp.kernel = P.kernel;
    kp.form = P.gradient_form;
    kp.phat_mode = phat_inline(c) ? (P.pressure_mode == 0 ? 1 : 2) : 0;
    kp.inv_re = c->r_n.inv_re;
    kp.inv_f = c->r_n.inv_f;
    kp.rho_s = c->rho_s;
    kp.sid = c->sid;
    kp.scn = c->scn;
    kp.pos_b = c->pos_b;
    kp.pos32 = c->pos32;
    kp.pos32lo = c->pos32lo;
    kp.vel32 = c->vel32;
    kp.g = c->grid;
    kp.st = c->st;
    if (P.precision == 1)
        k_gradient<true><<<nb, kBT, 0, c->stream>>>(n, c->type, c->pos_star, c->pos32_star, c->vel_star,
                                                    c->p, c->phat, c->nb_n_col, c->nb_n_cnt, c->cap_n,
                                                    c->r_n.re, c->r_n.re_f, c->coef_grad, P.dt, P.rho,
                                                    c->pos, c->vel, c->rows_f, c->scan_f + c->n, kp);
    else
        k_gradient<false><<<nb, kBT, 0, c->stream>>>(n, c->type, c->pos_star, c->pos32_star, c->vel_star,
                                                     c->p, c->phat, c->nb_n_col, c->nb_n_cnt, c->cap_n,
                                                     c->r_n.re, c->r_n.re_f, c->coef_grad, P.dt, P.rho,
                                                     c->pos, c->vel, c->rows_f, c->scan_f + c->n, kp);
    // the other particles keep r = r*, u = u*: their r*, u* are copies of r, u (walls and
    // dummies do not move), so there is nothing to write back
    c->launches += 1;
}

void launch_unpermute(Ctx* c, double* d_pos, double* d_vel, double* d_p, double* d_nstar,
                      uint8_t* d_flags, int8_t* d_types) {
    const int n = (int)c->n;
    k_unpermute<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->dim, c->id, c->pos, c->vel, c->p,
                                                             c->nstar, c->flag, c->type, d_pos, d_vel,
                                                             d_p, d_nstar, d_flags, d_types);
    c->launches += 1;
}

void launch_gather_props(Ctx* c) {
    if (!c->rho_id && !c->nu_id && !c->sid_id) return;
    const int n = (int)c->n;
    k_gather_props<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->id, c->rho_id, c->nu_id,
                                                               c->rho_s, c->nu_s, c->rho_ff,
                                                               c->sid_id, c->sid);
    c->launches += 1;
}

void launch_unpermute_u32(Ctx* c, const uint32_t* in, uint32_t* out) {
    const int n = (int)c->n;
    k_unpermute_u32<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->id, in, out);
    c->launches += 1;
}

void launch_ingest(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types,
                   bool keep_vel, bool keep_types) {
    const int n = (int)c->n;
    k_ingest<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->dim, d_pos, d_vel, d_types, c->pos,
                                                          c->vel, c->type, c->id, c->p, c->nstar,
                                                          c->flag, keep_vel ? 1 : 0,
                                                          keep_types ? 1 : 0, c->grid, c->pos32,
                                                          c->pos32lo);
    c->launches += 1;
}

void launch_same_state(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types) {
    const int n = (int)c->n;
    k_same_state<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->dim, d_pos, d_vel, d_types,
                                                             c->pos, c->vel, c->type, c->id, c->st);
    c->launches += 1;
}

void launch_check_stage(Ctx* c, const double* d_pos, const double* d_vel, const int8_t* d_types) {
    const int n = (int)c->n;
    k_check_stage<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(n, c->dim, d_pos, d_vel, d_types, c->st);
    c->launches += 1;
}

}  // namespace mps
