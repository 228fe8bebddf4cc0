// rows.cu -- per-particle pair sums over the step's candidate (Verlet) lists, one warp per
// particle: the lanes split the particle's candidates, so the pair arithmetic runs with
// (nearly) full warps whatever the hit pattern.
//
// The candidate list of particle i holds every j whose FP32 distance at r^k is below
// h = max(re_n, re_lap)(1 + s) (plus the FP32 rounding margin).  A pair closer than re_lap
// at r^k, or closer than max(re) at r* = r^k + dt u*, is in it as long as no particle moves
// more than s max(re)/2 in the step (checked; MPS_ESKIN otherwise).  Every use re-decides
// the exact predicate r^2 < re^2 in binary64 where the FP32 distance is inside the band.
//
//   predict (r^k, re_lap, FLUID rows):  u* = u + dt (nu lap(u) + g)  (Eq. 2 without the
//            pressure term; lap by Eq. 7), r* = r + dt u*.
//   build   (r*, all non-ghost rows):   n* (Eq. 5, re_n, every kind), free surface (Eq. 15),
//            PPE row: b (Eq. 13), c_ij = 2d/(n0 lambda rho) w (non-dummy j within re_lap;
//            PPE listing (Listing 2) of Sec. 4.3), diagonal sum c_ij + alpha_c/dt^2, compacted neighbour
//            lists for the PPE and for the gradient (non-dummy j within re_n), and the
//            equation-of-state pressure (Eq. 16).
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 256;

__device__ __forceinline__ float dist2_f(const float4& a, const float4& b) {
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ int kind_of(const float4& q) { return __float_as_int(q.w) & 0xff; }

struct PredictRows {
    int n, cap_v;
    const int32_t* vcol;
    const int32_t* vcnt;
    const float4* pos32;
    const double4* pos;
    const double4* vel;
    const float4* vel32;
    const int8_t* type;
    double4* pos_star;
    double4* vel_star;
    float4* pos32_star;
    DevStatus* st;
    Radius r;
    float tiny2;
    double coef_lap, nu, dt, g0, g1, g2, bmin0, bmin1, bmin2;
};

template <bool MIXED>
__global__ void __launch_bounds__(kBT) k_predict_rows(PredictRows a) {
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * kBT + threadIdx.x) >> 5, nw = (gridDim.x * kBT) >> 5;
    double dmax = 0.0;
    for (int i = gw; i < a.n; i += nw) {
        if (a.type[i] != kFluid) continue;
        const float4 pi32 = a.pos32[i];
        const double4 pi = a.pos[i];
        const double4 ui = a.vel[i];
        const float4 ui32 = make_float4((float)ui.x, (float)ui.y, (float)ui.z, 0.f);
        const int cnt = a.vcnt[i];
        const size_t base = (size_t)i * a.cap_v;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        float f0 = 0.f, f1 = 0.f, f2 = 0.f;
        for (int k = lane; k < cnt; k += 32) {
            const int j = a.vcol[base + k];
            const float r2 = dist2_f(pi32, a.pos32[j]);
            if (!in_radius(r2, a.r, a.pos, i, j, pi)) continue;
            if (MIXED && r2 >= a.tiny2) {
                const float w = fmaf(a.r.re_f, rsqrtf(r2), -1.f);
                const float4 uj = a.vel32[j];
                f0 = fmaf(uj.x - ui32.x, w, f0);
                f1 = fmaf(uj.y - ui32.y, w, f1);
                f2 = fmaf(uj.z - ui32.z, w, f2);
            } else {
                const double4 pj = a.pos[j];
                const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const double rr2 = fma(dz, dz, fma(dy, dy, dx * dx));
                if (!(rr2 > 0.0)) {
                    atomicOr(&a.st->err, kErrCoincident);
                    continue;
                }
                const double w = fma(a.r.re, rsqrt(rr2), -1.0);
                const double4 uj = a.vel[j];
                s0 = fma(uj.x - ui.x, w, s0);
                s1 = fma(uj.y - ui.y, w, s1);
                s2 = fma(uj.z - ui.z, w, s2);
            }
        }
        s0 = warp_sum(s0 + (double)f0);
        s1 = warp_sum(s1 + (double)f1);
        s2 = warp_sum(s2 + (double)f2);
        if (lane == 0) {
            // u* = u + dt (nu lap(u) + g); r* = r + dt u*  (one rounding per operation)
            const double l0 = a.coef_lap * s0, l1 = a.coef_lap * s1, l2 = a.coef_lap * s2;
            double4 us, ps;
            us.x = __dadd_rn(ui.x, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(a.nu, l0), a.g0)));
            us.y = __dadd_rn(ui.y, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(a.nu, l1), a.g1)));
            us.z = __dadd_rn(ui.z, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(a.nu, l2), a.g2)));
            us.w = 0.0;
            ps.x = __dadd_rn(pi.x, __dmul_rn(a.dt, us.x));
            ps.y = __dadd_rn(pi.y, __dmul_rn(a.dt, us.y));
            ps.z = __dadd_rn(pi.z, __dmul_rn(a.dt, us.z));
            ps.w = 0.0;
            a.vel_star[i] = us;
            a.pos_star[i] = ps;
            a.pos32_star[i] = make_float4((float)(ps.x - a.bmin0), (float)(ps.y - a.bmin1),
                                          (float)(ps.z - a.bmin2), pi32.w);
            const double dx = ps.x - pi.x, dy = ps.y - pi.y, dz = ps.z - pi.z;
            dmax = fmax(dmax, sqrt(dx * dx + dy * dy + dz * dz));
        }
    }
    if (lane == 0 && dmax > 0.0)
        atomicMax(&a.st->max_disp_bits, (unsigned long long)__double_as_longlong(dmax));
}

struct BuildRows {
    int n, cap_v, cap, cap_n, pressure_mode;
    const int32_t* vcol;
    const int32_t* vcnt;
    const float4* pos32;   // r*
    const double4* pos;    // r*
    const int8_t* type;
    DevStatus* st;
    Radius rn, rl;
    double coef_ppe, n0, beta, inv_dt2, diag_add, wc_k, gamma;
    int32_t* lap_col;
    double* lap_v64;
    float* lap_v32;
    int32_t* lap_cnt;
    int32_t* n_col;
    int32_t* n_cnt;
    double* nstar;
    uint8_t* flag;
    double* bvec;
    double* diag;
    double* p;
};

__global__ void __launch_bounds__(kBT) k_build_rows(BuildRows a) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int gw = (blockIdx.x * kBT + threadIdx.x) >> 5, nw = (gridDim.x * kBT) >> 5;
    unsigned n_surf = 0, n_ppe = 0;
    for (int i = gw; i < a.n; i += nw) {
        const int ti = a.type[i];
        if (ti == kGhost) continue;
        const bool rows = (ti == kFluid || ti == kWall);
        const float4 pi32 = a.pos32[i];
        const double4 pi = a.pos[i];
        const int cnt = a.vcnt[i];
        const size_t base = (size_t)i * a.cap_v;
        const size_t lbase = (size_t)i * a.cap, nbase = (size_t)i * a.cap_n;
        double nd = 0.0, dg = 0.0;
        int out_l = 0, out_n = 0;
        for (int kb = 0; kb < cnt; kb += 32) {
            const int k = kb + lane;
            bool inl = false, inn = false;
            int j = 0, kj = kDummy;
            double rs = 0.0;
            if (k < cnt) {
                j = a.vcol[base + k];
                const float4 q = a.pos32[j];
                kj = kind_of(q);
                const float r2 = dist2_f(pi32, q);
                inl = in_radius(r2, a.rl, a.pos, i, j, pi);
                inn = in_radius(r2, a.rn, a.pos, i, j, pi);
                if (inl || inn) {
                    const double4 pj = a.pos[j];
                    const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const double rr2 = fma(dz, dz, fma(dy, dy, dx * dx));
                    if (!(rr2 > 0.0)) {
                        atomicOr(&a.st->err, kErrCoincident);
                        inl = inn = false;
                    } else {
                        rs = rsqrt(rr2);
                    }
                }
            }
            if (inn) nd += fma(a.rn.re, rs, -1.0);
            const bool emit_l = rows && inl && kj != kDummy;
            const bool emit_n = rows && inn && kj != kDummy;
            double cij = 0.0;
            if (emit_l) {
                cij = a.coef_ppe * fma(a.rl.re, rs, -1.0);
                dg += cij;
            }
            const unsigned bl = __ballot_sync(0xffffffffu, emit_l);
            const unsigned bn = __ballot_sync(0xffffffffu, emit_n);
            if (emit_l) {
                const int q = out_l + __popc(bl & lt);
                if (q < a.cap) {
                    a.lap_col[lbase + q] = j;
                    a.lap_v64[lbase + q] = cij;
                    if (a.lap_v32) a.lap_v32[lbase + q] = (float)cij;
                }
            }
            if (emit_n) {
                const int q = out_n + __popc(bn & lt);
                if (q < a.cap_n) a.n_col[nbase + q] = j;
            }
            out_l += __popc(bl);
            out_n += __popc(bn);
        }
        nd = warp_sum(nd);
        dg = warp_sum(dg);
        if (lane == 0) {
            const bool surf = rows && (nd < a.beta * a.n0);
            const bool ppe = rows && !surf;
            a.nstar[i] = nd;
            a.flag[i] = surf ? 1 : 0;
            a.bvec[i] = ppe ? a.inv_dt2 * ((nd - a.n0) / a.n0) : 0.0;
            a.diag[i] = ppe ? dg + a.diag_add : 0.0;
            a.lap_cnt[i] = min(out_l, a.cap);
            a.n_cnt[i] = min(out_n, a.cap_n);
            if (out_l > a.cap || out_n > a.cap_n) atomicOr(&a.st->err, kErrCap);
            if (a.pressure_mode == 1) a.p[i] = ppe ? a.wc_k * (pow(nd / a.n0, a.gamma) - 1.0) : 0.0;
            n_surf += surf ? 1u : 0u;
            n_ppe += ppe ? 1u : 0u;
        }
    }
    if (lane == 0) {
        if (n_surf) atomicAdd(&a.st->n_surface, n_surf);
        if (n_ppe) atomicAdd(&a.st->n_ppe, n_ppe);
    }
}
}  // namespace

void launch_predict_rows(Ctx* c) {
    const mps_params& P = c->prm;
    PredictRows a;
    a.n = (int)c->n;
    a.cap_v = c->cap_v;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.pos32 = c->pos32;
    a.pos = c->pos;
    a.vel = c->vel;
    a.vel32 = c->vel32;
    a.type = c->type;
    a.pos_star = c->pos_star;
    a.vel_star = c->vel_star;
    a.pos32_star = c->pos32_star;
    a.st = c->st;
    a.r = c->r_lap;
    a.tiny2 = (float)(1e-6 * c->r_lap.re2);
    a.coef_lap = c->coef_lap;
    a.nu = P.nu;
    a.dt = P.dt;
    a.g0 = P.g[0];
    a.g1 = P.g[1];
    a.g2 = c->dim == 3 ? P.g[2] : 0.0;
    a.bmin0 = c->grid.bmin[0];
    a.bmin1 = c->grid.bmin[1];
    a.bmin2 = c->grid.bmin[2];
    const int grid = c->sms * 8;
    if (P.precision == 1) k_predict_rows<true><<<grid, kBT, 0, c->stream>>>(a);
    else k_predict_rows<false><<<grid, kBT, 0, c->stream>>>(a);
    c->launches += 1;
}

void launch_build_rows(Ctx* c) {
    const mps_params& P = c->prm;
    BuildRows a;
    a.n = (int)c->n;
    a.cap_v = c->cap_v;
    a.cap = c->cap;
    a.cap_n = c->cap_n;
    a.pressure_mode = P.pressure_mode;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.pos32 = c->pos32_star;
    a.pos = c->pos_star;
    a.type = c->type;
    a.st = c->st;
    a.rn = c->r_n;
    a.rl = c->r_lap;
    a.coef_ppe = c->coef_ppe;
    a.n0 = c->n0_pnd;
    a.beta = P.beta;
    a.inv_dt2 = c->inv_dt2;
    a.diag_add = c->diag_add;
    a.wc_k = P.rho * P.c0 * P.c0 / P.gamma;
    a.gamma = P.gamma;
    a.lap_col = c->nb_lap_col;
    a.lap_v64 = c->nb_lap_v64;
    a.lap_v32 = c->nb_lap_v32;
    a.lap_cnt = c->nb_lap_cnt;
    a.n_col = c->nb_n_col;
    a.n_cnt = c->nb_n_cnt;
    a.nstar = c->nstar;
    a.flag = c->flag;
    a.bvec = c->bvec;
    a.diag = c->diag;
    a.p = c->p;
    k_build_rows<<<c->sms * 8, kBT, 0, c->stream>>>(a);
    c->launches += 1;
}

}  // namespace mps
