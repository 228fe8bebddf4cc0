// adjoint.cu -- reverse of one step: the vector-Jacobian product of the step map
//   (r^k, u^k, g) -> (r^{k+1}, u^{k+1})
// for the PPE path (Eq. 13, Listing 2's assembly, CG) and the equation-of-state path
// (Eq. 16), with the kernel of Eq. 4, the difference-form gradient and one or two phases.
// Neighbour sets, the GHOST and free-surface sets, the clamp's active set and the particle
// that gives p_hat_i are held at the values of the forward step, within which the step is
// smooth; the reverse is its exact derivative (to the adjoint CG's tolerance).
//
// Notation: x = r_j - r_i, s = |x|, w(s) = re/s - 1, w'(s) = -re/s^2.  Every pair term of
// the forward adds a vector X to particle j's cotangent and -X to particle i's.  Here the
// sums run as gathers: row k visits its candidate list once per stage and adds the terms
// of the pairs (k, j) in which it plays either part, so nothing is scattered and every
// row's sum has a fixed order.  Stages, from the last forward stage back:
//   grad    (FLUID rows)  gG_i = -(dt/rho_i)(gu_i + dt gr_i), the cotangent of the pressure
//           gradient G_i = d/n0 sum_j (p_j - p_hat_i) x w/s^2 (non-dummy j, re_n, at r*);
//           gphat_i = -d/n0 gG_i . sum_j x w/s^2, and the minimiser of p_hat_i;
//   pbar    (FLUID/WALL)  gp_j = sum_i d/n0 (x . gG_i) w/s^2 + the p_hat cotangents of the
//           rows whose minimum is p_j, zero where p_j is not a function of the state (off
//           the PPE, or clamped); the equation of state turns it into gn*_j directly;
//   adjoint CG           A lam = gp on the same symmetric matrix (the PPE path);
//   star    (all kinds)   gr*_k: number density (every non-GHOST pair within re_n at r*)
//           and the gradient's pair terms over the step's gradient lists (DUMMY neighbours
//           from the candidate walk); PPE coefficients c_ij = K_ij w (non-dummy pairs
//           within re_lap, gc_ij = -lam_i (p_i - p_j) with the solution before the clamp)
//           over the step's stored PPE rows, whose stored c_ij give K re/s^3 =
//           (c + K)^3/(K re)^2; gu*_k = gu_k + dt gr*_k;
//   visc    (all kinds)   the prediction u* = u + dt (nu lap(u) + g) at r^k: the
//           Laplacian's transpose onto the velocities and its derivative in positions.
// All arithmetic is binary64.  Neighbour sets are decided by the same exact predicate as
// the forward kernels (FP32 band, binary64 inside it).
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 128;

__device__ __forceinline__ float dist2_f(const float4& a, const float4& b) {
    const float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ double dot3(const double4& a, const double4& b) {
    return fma(a.z, b.z, fma(a.y, b.y, a.x * b.x));
}
__device__ __forceinline__ double4 axpy4(double a, const double4& x, const double4& y) {
    return make_double4(fma(a, x.x, y.x), fma(a, x.y, y.y), fma(a, x.z, y.z), 0.0);
}
__device__ __forceinline__ double4 sub4(const double4& a, const double4& b) {
    return make_double4(a.x - b.x, a.y - b.y, a.z - b.z, 0.0);
}

struct AdjArgs {
    int n, cap, cap_n, cap_v, ppe, clamp, dim;
    const int8_t* type;
    const int32_t* id;
    const double4 *pos, *vel, *ps;     // r^k, u^k, r*
    const float4 *pos32, *ps32;        // FP32 copies (relative to the grid origin)
    const double *p, *phat, *ppre, *nstar, *diag;
    const uint8_t* flag;
    const int32_t *vcol, *vcnt, *ncol, *ncnt;
    const int32_t *lcol, *lcnt;        // the step's PPE rows: non-dummy j within re_lap at r*
    const double* lv64;                // with c_ij in binary64 (FP64 mode) or
    const float *lv32, *lvlo;          //   as float-float hi + lo (mixed mode)
    const double *rho_s, *nu_s;        // two-phase (null: uniform)
    Radius rn, rl;
    double n0, coef_grad, coef_ppe, coef_lap, rho, nu, dt, c0, gamma;
    double inv_n0dt2;                  // 1 / (n0 dt^2)
    // cotangents and work arrays (slot order)
    const double4 *gr, *gu;            // of r^{k+1}, u^{k+1}
    double4 *gG, *grs, *gus, *out_r, *out_u;
    double *gphat, *pbar, *lam, *gn;
    int32_t* amin;
    const uint8_t* was_ghost;          // by particle id
    double* gnu;                       // dL/dnu of every slot
};

__device__ __forceinline__ double rho_of(const AdjArgs& a, int i) { return a.rho_s ? a.rho_s[i] : a.rho; }
__device__ __forceinline__ double nu_of(const AdjArgs& a, int i) { return a.nu_s ? a.nu_s[i] : a.nu; }

// gradient stage: gG, gphat and the p_hat minimiser of every FLUID row
__global__ void __launch_bounds__(kBT) k_adj_grad(AdjArgs a) {
    const int i = blockIdx.x * kBT + threadIdx.x;
    if (i >= a.n) return;
    double4 gG = make_double4(0.0, 0.0, 0.0, 0.0);
    double gph = 0.0;
    int am = i;
    if (a.type[i] == kFluid) {
        gG = axpy4(a.dt, a.gr[i], a.gu[i]);
        const double k = -(a.dt / rho_of(a, i));
        gG = make_double4(k * gG.x, k * gG.y, k * gG.z, 0.0);
        const double4 pi = a.ps[i];
        double m = a.p[i];
        double4 S = make_double4(0.0, 0.0, 0.0, 0.0);
        const int cnt = a.ncnt[i];
        for (int t = 0; t < cnt; t++) {
            const int j = a.ncol[sell8(i, t, a.cap_n)];
            const double4 x = sub4(a.ps[j], pi);
            const double rs = rsqrt(dot3(x, x));
            const double q = fma(a.rn.re, rs, -1.0) * (rs * rs);   // w / s^2
            S = axpy4(q, x, S);
            if (a.ppe) {
                const double pj = a.p[j];
                if (pj < m) {
                    m = pj;
                    am = j;
                }
            }
        }
        gph = -a.coef_grad * dot3(gG, S);
    }
    a.gG[i] = gG;
    a.gphat[i] = gph;
    a.amin[i] = am;
}

// pressure cotangent of every FLUID/WALL row (zero where p does not depend on the state);
// the equation of state also gives the number-density cotangent
__global__ void __launch_bounds__(kBT) k_adj_pbar(AdjArgs a) {
    const int j = blockIdx.x * kBT + threadIdx.x;
    if (j >= a.n) return;
    const int tj = a.type[j];
    double pb = 0.0;
    bool live = false;
    if (tj == kFluid || tj == kWall) {
        if (tj == kFluid && a.amin[j] == j) pb += a.gphat[j];
        const double4 pj = a.ps[j];
        const int cnt = a.ncnt[j];
        for (int t = 0; t < cnt; t++) {
            const int i = a.ncol[sell8(j, t, a.cap_n)];
            if (a.type[i] != kFluid) continue;
            const double4 x = sub4(pj, a.ps[i]);   // r_j - r_i for the pair (i, j) of row i
            const double rs = rsqrt(dot3(x, x));
            const double q = fma(a.rn.re, rs, -1.0) * (rs * rs);
            pb = fma(a.coef_grad * q, dot3(x, a.gG[i]), pb);
            if (a.amin[i] == j) pb += a.gphat[i];
        }
        live = a.ppe ? (a.diag[j] != 0.0 && (!a.clamp || a.ppre[j] > 0.0)) : (a.flag[j] == 0);
    }
    if (!live) pb = 0.0;
    a.pbar[j] = pb;
    if (!a.ppe) {
        a.gn[j] = live ? pb * rho_of(a, j) * a.c0 * a.c0 * pow(a.nstar[j] / a.n0, a.gamma - 1.0) / a.n0
                       : 0.0;
    }
}

// the PPE path's number-density cotangent from the adjoint solution
__device__ __forceinline__ double gn_of(const AdjArgs& a, int i) {
    if (!a.ppe) return a.gn[i];
    return a.diag[i] != 0.0 ? a.lam[i] * a.inv_n0dt2 : 0.0;
}

// cotangent of r* (and u* of FLUID rows): number density, PPE coefficients, gradient pairs.
// On GB300 an FP64 warp instruction costs the same whatever the number of active lanes, so
// the pair loops run over dense lists wherever the forward step stored them: FLUID / WALL
// rows (the bucket build's list of them, one thread each) take their non-dummy neighbours
// within re_n from the gradient list and their PPE pairs from the PPE rows; only the DUMMY
// neighbours (number density alone) come from the candidate walk.
__global__ void __launch_bounds__(kBT) k_adj_star_fw(AdjArgs a, const int32_t* rows,
                                                     const uint32_t* nrows, double inv_kre2) {
    const int tid = blockIdx.x * kBT + threadIdx.x;
    if (tid >= (int)*nrows) return;
    const int k = rows[tid];
    const bool fk = a.type[k] == kFluid;
    double4 acc = a.gr[k];
    const double gnk = gn_of(a, k);
    const double pk = a.p[k], phk = a.phat[k];
    const double4 gGk = a.gG[k];
    const double4 xk = a.ps[k];
    // non-dummy pairs within re_n: number density and the gradient's pair terms
    const int cn = a.ncnt[k];
    for (int t = 0; t < cn; t++) {
        const int j = a.ncol[sell8(k, t, a.cap_n)];
        const double4 x = sub4(a.ps[j], xk);
        // every power of 1/s from one reciprocal square root
        const double rs = rsqrt(dot3(x, x));
        const double rs2 = rs * rs;
        const double is3 = rs2 * rs;
        // n*_k and n*_j both hold w(s): -(gn_k + gn_j) w'(s) x/s
        acc = axpy4((gnk + gn_of(a, j)) * a.rn.re * is3, x, acc);
        const double w = fma(a.rn.re, rs, -1.0);
        const double q = w * rs2;
        // (d/ds (w/s^2)) / s = -re/s^5 - 2 w/s^4
        const double qds = -rs2 * rs2 * fma(a.rn.re, rs, 2.0 * w);
        if (fk) {   // pair (k, j) of row k's gradient: -X
            const double dg = dot3(x, gGk);
            const double f = a.coef_grad * (a.p[j] - phk);
            acc = axpy4(-f * q, gGk, acc);
            acc = axpy4(-f * qds * dg, x, acc);
        }
        if (a.type[j] == kFluid) {   // pair (j, k) of row j's gradient: +X
            const double4 gGj = a.gG[j];
            const double dg = dot3(x, gGj);
            const double f = a.coef_grad * (pk - a.phat[j]);
            acc = axpy4(f * q, gGj, acc);
            acc = axpy4(f * qds * dg, x, acc);
        }
    }
    // DUMMY neighbours within re_n (their n* enters no equation): -gn_k w'(s) x/s
    if (gnk != 0.0) {
        const float4 qk = a.ps32[k];
        const int cnt = a.vcnt[k];
        for (int t = 0; t < cnt; t++) {
            const int j = a.vcol[sell8(k, t, a.cap_v)];
            if (a.type[j] != kDummy) continue;
            if (!in_radius(dist2_f(qk, a.ps32[j]), a.rn, a.ps, k, j, xk)) continue;
            const double4 x = sub4(a.ps[j], xk);
            const double rs = rsqrt(dot3(x, x));
            acc = axpy4(gnk * a.rn.re * (rs * rs * rs), x, acc);
        }
    }
    // PPE coefficient pairs (non-dummy j within re_lap): the row's stored coefficients.
    // -(gc_kj + gc_jk) K w'(s) x/s = (p_k - p_j)(lam_j - lam_k) K re/s^3 x, and with
    // c = K (re/s - 1) stored, K re/s^3 = (c + K)^3 / (K re)^2: no square root
    if (a.ppe) {
        const bool rk = a.diag[k] != 0.0;
        const double lamk = rk ? a.lam[k] : 0.0, ppk = rk ? a.ppre[k] : 0.0;
        const double rhok = a.rho_s ? a.rho_s[k] : 0.0;
        const int m = a.lcnt[k];
        for (int t = 0; t < m; t++) {
            const size_t q = sell8(k, t, a.cap);
            const int j = a.lcol[q];
            const double c = a.lv64 ? a.lv64[q] : (double)a.lv32[q] + (double)a.lvlo[q];
            const bool rj = a.diag[j] != 0.0;
            const double lamj = rj ? a.lam[j] : 0.0, ppj = rj ? a.ppre[j] : 0.0;
            double K = a.coef_ppe, ik = inv_kre2;
            if (a.rho_s) {   // two-phase pair factor
                K = a.coef_lap * (2.0 / (rhok + a.rho_s[j]));
                const double kre = K * a.rl.re;
                ik = 1.0 / (kre * kre);
            }
            const double u = c + K;
            const double f = (ppk - ppj) * (lamj - lamk) * (u * u * u * ik);
            acc = axpy4(f, sub4(a.ps[j], xk), acc);
        }
    }
    a.grs[k] = acc;
    a.gus[k] = fk ? axpy4(a.dt, acc, a.gu[k]) : make_double4(0.0, 0.0, 0.0, 0.0);
}

// DUMMY rows (number density of their FLUID / WALL neighbours within re_n) and GHOST rows
// (carried through); FLUID / WALL slots are left to k_adj_star_fw
__global__ void __launch_bounds__(kBT) k_adj_star_other(AdjArgs a) {
    const int k = blockIdx.x * kBT + threadIdx.x;
    if (k >= a.n) return;
    const int tk = a.type[k];
    if (tk == kFluid || tk == kWall) return;
    double4 acc = a.gr[k];
    if (tk == kDummy) {
        const double4 xk = a.ps[k];
        const float4 qk = a.ps32[k];
        const int cnt = a.vcnt[k];
        for (int t = 0; t < cnt; t++) {
            const int j = a.vcol[sell8(k, t, a.cap_v)];
            if (!in_radius(dist2_f(qk, a.ps32[j]), a.rn, a.ps, k, j, xk)) continue;
            const double gnj = gn_of(a, j);
            if (gnj == 0.0) continue;
            const double4 x = sub4(a.ps[j], xk);
            const double rs = rsqrt(dot3(x, x));
            acc = axpy4(gnj * a.rn.re * (rs * rs * rs), x, acc);
        }
    }
    a.grs[k] = acc;
    a.gus[k] = make_double4(0.0, 0.0, 0.0, 0.0);
}

// prediction at r^k: the Laplacian's transpose and its position derivative; final
// cotangents.  Only pairs with a FLUID end carry viscosity terms, so FLUID rows (the bucket
// build's list of them) and the other rows run as two kernels, and the other rows skip
// non-FLUID candidates before any binary64 work.
//   pair (k, j), x = r_j - r_k, a_k = dt nu_k 2d/(n0 lambda) gu*_k (0 unless k is FLUID):
//   gu_k += w (a_j - a_k),  gr_k -= w'(s)/s ((a_k - a_j) . (u_j - u_k)) x
// The viscosity enters u*_k linearly: dL/dnu_k = dt 2d/(n0 lambda) sum_j w (gu*_k . (u_j - u_k))
// for FLUID k; FLUID rows return w to sum it.
__device__ __forceinline__ double visc_pair(const AdjArgs& a, int j, const double4& xk,
                                            const double4& uk, const double4& ak, double4& orr,
                                            double4& ou) {
    const double4 x = sub4(a.pos[j], xk);
    const double rs = rsqrt(dot3(x, x));
    const double w = fma(a.rl.re, rs, -1.0);
    const double wd_s = -a.rl.re * (rs * rs * rs);   // w'(s)/s
    double4 aj = make_double4(0.0, 0.0, 0.0, 0.0);
    if (a.type[j] == kFluid) {
        const double kj = a.dt * nu_of(a, j) * a.coef_lap;
        const double4 gsj = a.gus[j];
        aj = make_double4(kj * gsj.x, kj * gsj.y, kj * gsj.z, 0.0);
    }
    const double4 da = sub4(aj, ak);
    ou = axpy4(w, da, ou);
    orr = axpy4(wd_s * dot3(da, sub4(a.vel[j], uk)), x, orr);
    return w;
}

__global__ void __launch_bounds__(kBT) k_adj_visc_f(AdjArgs a, const int32_t* rows,
                                                    const uint32_t* nrows) {
    const int tid = blockIdx.x * kBT + threadIdx.x;
    if (tid >= (int)*nrows) return;
    const int k = rows[tid];
    double4 orr = a.grs[k];
    const double4 gsk = a.gus[k];
    double4 ou = gsk;
    const double kk = a.dt * nu_of(a, k) * a.coef_lap;
    const double4 ak = make_double4(kk * gsk.x, kk * gsk.y, kk * gsk.z, 0.0);
    const double4 xk = a.pos[k], uk = a.vel[k];
    const float4 qk = a.pos32[k];
    const int cnt = a.vcnt[k];
    double lap = 0.0;   // sum_j w (gu*_k . (u_j - u_k))
    for (int t = 0; t < cnt; t++) {
        const int j = a.vcol[sell8(k, t, a.cap_v)];
        if (!in_radius(dist2_f(qk, a.pos32[j]), a.rl, a.pos, k, j, xk)) continue;
        const double w = visc_pair(a, j, xk, uk, ak, orr, ou);
        lap = fma(w, dot3(gsk, sub4(a.vel[j], uk)), lap);
    }
    a.out_r[k] = orr;
    a.out_u[k] = ou;
    a.gnu[k] = a.dt * a.coef_lap * lap;
}

__global__ void __launch_bounds__(kBT) k_adj_visc_other(AdjArgs a) {
    const int k = blockIdx.x * kBT + threadIdx.x;
    if (k >= a.n) return;
    const int tk = a.type[k];
    if (tk == kFluid) return;
    a.gnu[k] = 0.0;   // the viscosity acts on FLUID particles only
    if (tk == kGhost) {
        a.out_r[k] = a.gr[k];
        a.out_u[k] = a.was_ghost[a.id[k]] ? a.gu[k] : make_double4(0.0, 0.0, 0.0, 0.0);
        return;
    }
    double4 orr = a.grs[k];
    double4 ou = a.gu[k];
    const double4 ak = make_double4(0.0, 0.0, 0.0, 0.0);
    const double4 xk = a.pos[k], uk = a.vel[k];
    const float4 qk = a.pos32[k];
    const int cnt = a.vcnt[k];
    for (int t = 0; t < cnt; t++) {
        const int j = a.vcol[sell8(k, t, a.cap_v)];
        if (a.type[j] != kFluid) continue;
        if (!in_radius(dist2_f(qk, a.pos32[j]), a.rl, a.pos, k, j, xk)) continue;
        visc_pair(a, j, xk, uk, ak, orr, ou);
    }
    a.out_r[k] = orr;
    a.out_u[k] = ou;
}

// dL/dg = dt sum over FLUID rows of gu*: per-block partial sums (gus is zero off FLUID
// rows), then one block adds them in block order
__global__ void __launch_bounds__(256) k_adj_gpart(int n, const double4* gus, double* part) {
    __shared__ double sm[8];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
        const double4 v = gus[i];
        s0 += v.x;
        s1 += v.y;
        s2 += v.z;
    }
    s0 = block_sum<256>(s0, sm);
    s1 = block_sum<256>(s1, sm);
    s2 = block_sum<256>(s2, sm);
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x] = s0;
        part[3 * blockIdx.x + 1] = s1;
        part[3 * blockIdx.x + 2] = s2;
    }
}

__global__ void __launch_bounds__(256) k_adj_gsum(int nb, const double* part, double dt, double* out) {
    __shared__ double sm[8];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += 256)
        for (int a = 0; a < 3; a++) s[a] += part[3 * b + a];
    for (int a = 0; a < 3; a++) {
        const double t = block_sum<256>(s[a], sm);
        if (threadIdx.x == 0) out[a] = dt * t;
    }
}

// was_ghost[id] of every particle before the step (the step may turn more into GHOSTs)
__global__ void k_adj_mark(int n, const int8_t* type, const int32_t* id, uint8_t* was_ghost) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n) was_ghost[id[s]] = type[s] == kGhost ? 1 : 0;
}

// caller's cotangents (original order, dim per particle) into slot order
__global__ void k_adj_load(int n, int dim, const int32_t* id, const double* gpos, const double* gvel,
                           double4* gr, double4* gu) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const size_t i = (size_t)id[s] * dim;
    double r[3] = {0.0, 0.0, 0.0}, u[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < dim; d++) {
        r[d] = gpos[i + d];
        u[d] = gvel[i + d];
    }
    gr[s] = make_double4(r[0], r[1], r[2], 0.0);
    gu[s] = make_double4(u[0], u[1], u[2], 0.0);
}

__global__ void k_adj_store(int n, int dim, const int32_t* id, const double4* r, const double4* u,
                            const double* gnu, double* o_r, double* o_u, double* o_nu) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (o_nu) o_nu[id[s]] = gnu[s];
    const size_t i = (size_t)id[s] * dim;
    const double4 a = r[s], b = u[s];
    const double ra[3] = {a.x, a.y, a.z}, ua[3] = {b.x, b.y, b.z};
    for (int d = 0; d < dim; d++) {
        o_r[i + d] = ra[d];
        o_u[i + d] = ua[d];
    }
}

AdjArgs adj_args(Ctx* c) {
    const mps_params& P = c->prm;
    AdjArgs a;
    a.n = (int)c->n;
    a.cap = c->cap;
    a.cap_n = c->cap_n;
    a.cap_v = c->cap_v;
    a.ppe = P.pressure_mode == 0;
    a.clamp = P.clamp_negative_p != 0;
    a.dim = c->dim;
    a.type = c->type;
    a.id = c->id;
    a.pos = c->pos;
    a.vel = c->vel;
    a.ps = c->pos_star;
    a.pos32 = c->pos32;
    a.ps32 = c->pos32_star;
    a.p = c->p;
    a.phat = c->phat;
    a.ppre = c->adj.ppre;
    a.nstar = c->nstar;
    a.diag = c->diag;
    a.flag = c->flag;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.ncol = c->nb_n_col;
    a.ncnt = c->nb_n_cnt;
    a.lcol = c->nb_lap_col;
    a.lcnt = c->nb_lap_cnt;
    a.lv64 = c->prm.precision == 0 ? c->nb_lap_v64 : nullptr;
    a.lv32 = c->nb_lap_v32;
    a.lvlo = c->nb_lap_vlo;
    a.rho_s = c->rho_s;
    a.nu_s = c->nu_s;
    a.rn = c->r_n;
    a.rl = c->r_lap;
    a.n0 = c->n0_pnd;
    a.coef_grad = c->coef_grad;
    a.coef_ppe = c->coef_ppe;
    a.coef_lap = c->coef_lap;
    a.rho = P.rho;
    a.nu = P.nu;
    a.dt = P.dt;
    a.c0 = P.c0;
    a.gamma = P.gamma;
    a.inv_n0dt2 = 1.0 / (c->n0_pnd * P.dt * P.dt);
    a.gr = c->adj.gr;
    a.gu = c->adj.gu;
    a.gG = c->adj.gG;
    a.grs = c->adj.grs;
    a.gus = c->adj.gus;
    a.out_r = c->adj.out_r;
    a.out_u = c->adj.out_u;
    a.gphat = c->adj.gphat;
    a.pbar = c->adj.pbar;
    a.lam = c->adj.lam;
    a.gn = c->adj.gn;
    a.amin = c->adj.amin;
    a.was_ghost = c->adj.was_ghost;
    a.gnu = c->adj.gnu;
    return a;
}

inline int blocks(int64_t n, int bt) { return (int)((n + bt - 1) / bt); }

}  // namespace

void launch_adj_mark(Ctx* c) {
    const int n = (int)c->n;
    k_adj_mark<<<blocks(n, 256), 256, 0, c->stream>>>(n, c->type, c->id, c->adj.was_ghost);
    c->launches += 1;
}

void launch_adj_load(Ctx* c, const double* d_gpos, const double* d_gvel) {
    const int n = (int)c->n;
    k_adj_load<<<blocks(n, 256), 256, 0, c->stream>>>(n, c->dim, c->id, d_gpos, d_gvel, c->adj.gr,
                                                       c->adj.gu);
    c->launches += 1;
}

void launch_adj_front(Ctx* c) {
    const AdjArgs a = adj_args(c);
    const int g = blocks(c->n, kBT);
    k_adj_grad<<<g, kBT, 0, c->stream>>>(a);
    k_adj_pbar<<<g, kBT, 0, c->stream>>>(a);
    c->launches += 2;
}

void launch_adj_back(Ctx* c, double* d_gsum) {
    const AdjArgs a = adj_args(c);
    const int g = blocks(c->n, kBT);
    const double kre = c->coef_ppe * c->r_lap.re;
    k_adj_star_fw<<<g, kBT, 0, c->stream>>>(a, c->rows_fw, c->scan_fw + c->n, 1.0 / (kre * kre));
    k_adj_star_other<<<g, kBT, 0, c->stream>>>(a);
    k_adj_visc_f<<<g, kBT, 0, c->stream>>>(a, c->rows_f, c->scan_f + c->n);
    k_adj_visc_other<<<g, kBT, 0, c->stream>>>(a);
    const int nb = std::min<int>(blocks(c->n, 256), 1024);   // c->partials holds 4096 doubles
    k_adj_gpart<<<nb, 256, 0, c->stream>>>((int)c->n, c->adj.gus, c->partials);
    k_adj_gsum<<<1, 256, 0, c->stream>>>(nb, c->partials, c->prm.dt, d_gsum);
    c->launches += 6;
}

void launch_adj_store(Ctx* c, double* d_out_r, double* d_out_u, double* d_out_nu) {
    const int n = (int)c->n;
    k_adj_store<<<blocks(n, 256), 256, 0, c->stream>>>(n, c->dim, c->id, c->adj.out_r,
                                                        c->adj.out_u, c->adj.gnu, d_out_r,
                                                        d_out_u, d_out_nu);
    c->launches += 1;
}

}  // namespace mps
