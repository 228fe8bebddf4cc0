// rows.cu -- per-particle pair sums over the step's candidate (Verlet) lists, one thread per
// particle.  Lists are sell8 (a row's entries in 32-byte groups, the 32 rows of a warp's
// slice side by side), and every per-particle FP64 operation (the state update, the PPE row) runs with all lanes of
// the warp busy: on GB300 an FP64 warp instruction costs the FP64 pipe ~64 cycles whatever
// the number of active lanes.
//
// The candidate list of particle i holds every j whose FP32 distance at r^k is below
// max(re_n, re_lap)(1 + s') (plus the FP32 rounding margin), s' <= s the list skin the
// recent motion needs (the cells keep the full skin s).  A pair closer than re_lap at r^k,
// or closer than max(re) at r* = r^k + dt u*, is in it as long as no particle moves more
// than s' max(re)/2 in the step (checked: the step is gathered again with the full skin,
// and MPS_ESKIN past that).
//
// Exact predicate r^2 < re^2 of the binary64 definition, in three tiers: the FP32 squared
// distance decides outside a band of its rounding error; inside it, a float-float distance
// decides outside a band ~1e-11 re^2 wide; the few pairs left (exact lattice geometry of
// unjittered walls) are decided in binary64 with ((dx*dx)+(dy*dy))+(dz*dz) < re*re.
//
//   predict (r^k, re_lap, FLUID):  u* = u + dt (nu lap(u) + g)  (Eq. 2 without the pressure
//            term; lap by Eq. 7), r* = r + dt u*.
//   build   (r*, FLUID and WALL particles):  n* (Eq. 5, re_n, neighbours of every kind), free surface
//            (Eq. 15), PPE row: b (Eq. 13), c_ij = 2d/(n0 lambda rho) w (non-dummy j within
//            re_lap; PPE listing (Listing 2) of Sec. 4.3), diagonal sum c_ij + alpha_c/dt^2,
//            neighbour lists for the PPE and the gradient (non-dummy j within re_n), and the
//            equation-of-state pressure (Eq. 16).
// Precision: FP64 mode evaluates pair terms in binary64; mixed mode evaluates the viscosity
// terms in FP32 (compensated FP32 sums, stored in binary64) and the number density
// and PPE coefficients in float-float (relative error ~1e-13), accumulated in float-float
// and stored in binary64.
#include "ff.cuh"
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 128;
// the build's blocks (defaults; params.build_block and the autotuner choose 64, 128 or 256):
// 256 rows of neighbouring particles share more of their candidates in L1 (5% faster than
// 128 on the 3D dam break; the prediction is faster at 128); the mixed build with the PPE
// takes 128, its output staging ring (RowStage) being deep
constexpr int kBuildBT = 256;
constexpr int kBuildRingBT = 128;

__device__ __forceinline__ float dist2_f(const float4& a, const float4& b) {
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ int kind_of(const float4& q) { return __float_as_int(q.w) & 0xff; }

// float-float squared distance from hi/lo coordinate pairs
__device__ __forceinline__ ff pair_r2(const float4& ih, const float4& il, const float4& jh,
                                     const float4& jl) {
    return ff_dist2(ff_diff(ih.x, il.x, jh.x, jl.x), ff_diff(ih.y, il.y, jh.y, jl.y),
                    ff_diff(ih.z, il.z, jh.z, jl.z));
}

// tier 2 and 3 of the predicate for a pair inside the FP32 band
__device__ __forceinline__ bool decide_band(const ff& r2, const Radius& r, const double4* pos,
                                            const double4& pi, int j) {
    const float d = (r2.h - r.re2_h) + (r2.l - r.re2_l);
    if (d <= -r.ff_tol) return true;
    if (d >= r.ff_tol) return false;
    return exact_dist2(pi, pos[j]) < r.re2;
}

// compensated summation (Kahan): s + (-e) carries the sum to about twice FP32 precision
__device__ __forceinline__ void kahan_add(float& s, float& e, float v) {
    const float y = v - e;
    const float t = s + y;
    e = (t - s) - y;
    s = t;
}

// 1 inside, 0 outside, from the FP32 distance; 2: needs the finer tiers
__device__ __forceinline__ int tier1(float r2, const Radius& r) {
    return r2 < r.lo ? 1 : (r2 >= r.hi ? 0 : 2);
}

struct PredictArgs {
    int n, cap_v;
    const int32_t* vcol;
    const int32_t* vcnt;
    const float4* pos32;
    const float4* pos32lo;
    const double4* pos;
    const double4* pos_b;   // where the candidate lists were gathered (r^k when gathered this step)
    const int32_t* rows;    // FLUID slots in slot order
    const uint32_t* nrows;  // their count
    const double* nu_s;     // two-phase: per-slot viscosity (null: nu)
    int kernel;             // 0: re/r - 1 (Eq. 4); 1: (1 - r/re)^3
    const uint16_t* sid;    // ensemble: scene of every slot
    const SceneParams* scn;
    const double4* vel;
    const float4* vel32;
    const int8_t* type;
    double4* pos_star;
    double4* vel_star;
    float4* pos32_star;
    float4* pff_star;   // r* again as (hi, lo) pairs: slot i at 2 i and 2 i + 1
    DevStatus* st;
    Radius r;
    double coef_lap, nu, dt, g0, g1, g2, bmin0, bmin1, bmin2;
    const double* g_dev;    // non-null: the acceleration is read here (a step graph's control block)
};

// MULTI: an ensemble, whose radii and coefficients are those of each row's scene.
// TPR threads per FLUID row (the bucket build's list of FLUID slots; adjacent lanes): thread
// t of a row takes the candidates t, t + TPR, ... of its list, so each walks a chain TPR
// times shorter; their sums are added across the lanes and the first one writes the row.
template <bool MIXED, bool MULTI, int TPR>
__global__ void __launch_bounds__(kBT) k_predict(PredictArgs a) {
    const int tid = blockIdx.x * kBT + threadIdx.x;
    const int row = tid / TPR, sub = tid % TPR;
    const int i = row < (int)*a.nrows ? a.rows[row] : -1;
    // the lanes of one row (valid or not together)
    const unsigned row_mask = TPR == 1 ? (1u << (threadIdx.x & 31))
                                       : (((1u << TPR) - 1u) << ((threadIdx.x & 31) & ~(TPR - 1)));
    double disp = 0.0;
    if (i >= 0) {
        Radius R = a.r;
        double coef_lap = a.coef_lap;
        if (MULTI) {
            const SceneParams& sp = a.scn[a.sid[i]];
            R = sp.rl;
            coef_lap = sp.coef_lap;
        }
        const float4 ih = a.pos32[i], il = a.pos32lo[i];
        // the binary64 state of i: held through the walk on the FP64 path; the mixed path
        // reads it in the rare binary64 tier and after the walk, which leaves it registers
        // for the neighbour's velocity in flight
        double4 pi = make_double4(0.0, 0.0, 0.0, 0.0), ui = pi;
        if (!MIXED) {
            pi = a.pos[i];
            ui = a.vel[i];
        }
        const float4 u32 = a.vel32[i];
        const int cnt = a.vcnt[i];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        // FP32 terms in compensated (Kahan) FP32 sums: value f, running correction e
        float f0 = 0.f, f1 = 0.f, f2 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f;
        // two-stage software pipeline: the slot two candidates ahead and the position of the
        // next one are in flight (this thread's candidates: sub, sub + TPR, ...)
        int jn = cnt > sub + TPR ? a.vcol[sell8(i, sub + TPR, a.cap_v)] : 0;
        int j0 = cnt > sub ? a.vcol[sell8(i, sub, a.cap_v)] : 0;
        float4 qn = a.pos32[j0];
        // mixed: the FP32 velocity of the next candidate is in flight with its position
        // (nearly every candidate is a member)
        float4 vn = MIXED ? a.vel32[j0] : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = sub; k < cnt; k += TPR) {
            const int j = j0;
            const float4 jh = qn;
            const float4 vj = vn;
            j0 = jn;
            if (k + TPR < cnt) {
                qn = a.pos32[jn];
                if (MIXED) vn = a.vel32[jn];
            }
            if (k + 2 * TPR < cnt) jn = a.vcol[sell8(i, k + 2 * TPR, a.cap_v)];
            const float r2 = dist2_f(ih, jh);
            int t = tier1(r2, R);
            if (t == 2)
                t = decide_band(pair_r2(ih, il, jh, a.pos32lo[j]), R, a.pos, MIXED ? a.pos[i] : pi, j) ? 1 : 0;
            if (!t) continue;
            if (MIXED) {
                if (!(r2 > 0.f)) {   // coincident to FP32: decide in binary64
                    if (!(exact_dist2(a.pos[i], a.pos[j]) > 0.0)) atomicOr(&a.st->err, kErrCoincident);
                    continue;
                }
                const float rs = rsqrtf(r2);
                const float w = a.kernel == 1 ? cubic_w_f(r2, rs, R.inv_f) : fmaf(R.re_f, rs, -1.f);
                const float4 uj = vj;
                kahan_add(f0, e0, (uj.x - u32.x) * w);
                kahan_add(f1, e1, (uj.y - u32.y) * w);
                kahan_add(f2, e2, (uj.z - u32.z) * w);
            } else {
                const double4 pj = a.pos[j];
                const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const double rr2 = fma(dz, dz, fma(dy, dy, dx * dx));
                if (!(rr2 > 0.0)) {
                    atomicOr(&a.st->err, kErrCoincident);
                    continue;
                }
                const double rs = rsqrt(rr2);
                const double w = a.kernel == 1 ? cubic_w_d(rr2, rs, R.inv_re) : fma(R.re, rs, -1.0);
                const double4 uj = a.vel[j];
                s0 = fma(uj.x - ui.x, w, s0);
                s1 = fma(uj.y - ui.y, w, s1);
                s2 = fma(uj.z - ui.z, w, s2);
            }
        }
        if (MIXED) {
            s0 = ff_to_double_fast({f0, -e0});
            s1 = ff_to_double_fast({f1, -e1});
            s2 = ff_to_double_fast({f2, -e2});
            pi = a.pos[i];
            ui = a.vel[i];
        }
        // the row's sums from its TPR threads (the same bits in each: a + b = b + a)
        for (int o = 1; o < TPR; o <<= 1) {
            s0 += __shfl_xor_sync(row_mask, s0, o);
            s1 += __shfl_xor_sync(row_mask, s1, o);
            s2 += __shfl_xor_sync(row_mask, s2, o);
        }
        // u* = u + dt (nu lap(u) + g); r* = r + dt u*  (one rounding per operation)
        const double l0 = coef_lap * s0, l1 = coef_lap * s1, l2 = coef_lap * s2;
        double4 us, ps;
        const double nu = a.nu_s ? a.nu_s[i] : a.nu;
        const double g0 = a.g_dev ? a.g_dev[0] : a.g0, g1 = a.g_dev ? a.g_dev[1] : a.g1,
                     g2 = a.g_dev ? a.g_dev[2] : a.g2;
        us.x = __dadd_rn(ui.x, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(nu, l0), g0)));
        us.y = __dadd_rn(ui.y, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(nu, l1), g1)));
        us.z = __dadd_rn(ui.z, __dmul_rn(a.dt, __dadd_rn(__dmul_rn(nu, l2), g2)));
        us.w = 0.0;
        ps.x = __dadd_rn(pi.x, __dmul_rn(a.dt, us.x));
        ps.y = __dadd_rn(pi.y, __dmul_rn(a.dt, us.y));
        ps.z = __dadd_rn(pi.z, __dmul_rn(a.dt, us.z));
        ps.w = 0.0;
        if (sub == 0) {
            a.vel_star[i] = us;
            a.pos_star[i] = ps;
            float4 h4, l4;
            split_rel(ps.x, a.bmin0, &h4.x, &l4.x);
            split_rel(ps.y, a.bmin1, &h4.y, &l4.y);
            split_rel(ps.z, a.bmin2, &h4.z, &l4.z);
            h4.w = ih.w;
            l4.w = 0.f;
            a.pos32_star[i] = h4;
            a.pff_star[2 * i] = h4;
            a.pff_star[2 * i + 1] = l4;
            const double4 pb = a.pos_b ? a.pos_b[i] : pi;
            const double dx = ps.x - pb.x, dy = ps.y - pb.y, dz = ps.z - pb.z;
            disp = fma(dz, dz, fma(dy, dy, dx * dx));   // squared; the host takes the root
        }
    }
    // warp max of the squared displacement (non-negative doubles order like their bits)
    unsigned long long v = (unsigned long long)__double_as_longlong(disp);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0 && v) atomicMax(&a.st->max_disp_bits, v);
}

struct BuildArgs {
    int n, cap_v, cap, cap_n, pressure_mode;
    const int32_t* rows;    // FLUID and WALL slots in slot order
    const uint32_t* nrows;  // their count
    // two-phase: per-slot density (FP64 and float-float) or null; the PPE coefficient then
    // takes coef0 = 2d/(n0 lambda) times the pair factor 2/(rho_i + rho_j)
    const double* rho_s;
    const float2* rho_ff;
    double coef0, wc_c;     // wc_c = c0^2/gamma
    int kernel;             // 0: re/r - 1 (Eq. 4); 1: (1 - r/re)^3
    int source;             // 0: Eq. 13; 1: HS (Eq. 21), from the predicted velocities
    const double4* vel_star;
    double dt;
    const double* ecs_nk;   // ECS: n^k and (Dn/Dt)^k per row (source 2)
    const double* ecs_dk;
    const uint16_t* sid;    // ensemble: scene of every slot
    const SceneParams* scn;
    const int32_t* vcol;
    const int32_t* vcnt;
    const float4* pos32;     // r*
    const float4* pff;       // r* as (hi, lo) pairs: one 32-byte sector per particle
    const double4* pos;      // r*
    const int8_t* type;
    DevStatus* st;
    Radius rn, rl;
    double coef_ppe, n0, beta, inv_dt2, diag_add, wc_k, gamma;
    ff cre_ff, ncoef_ff;   // coef_ppe * re_lap and -coef_ppe as float-float
    int32_t* lap_col;
    double* lap_v64;   // FP64 mode
    float* lap_v32;    // mixed mode: hi part (the FP32 coefficient)
    float* lap_vlo;    // mixed mode: lo part
    int32_t* lap_cnt;
    int32_t* n_col;
    int32_t* n_cnt;
    double* nstar;
    uint8_t* flag;
    double* bvec;
    double* diag;
    float* diag32;
    double* p;
};

// One HS source term (Eq. 21) in binary64: re / r^3 (r_ij . (u*_j - u*_i)) with the offset
// and 1/r given as float-float (converted by bit moves plus one addition)
__device__ __forceinline__ double hs_term(ff dx, ff dy, ff dz, ff y, const double4& uj,
                                          const double4& ui, double re) {
    const double x = ff_to_double_fast(dx), yy = ff_to_double_fast(dy), z = ff_to_double_fast(dz);
    const double ry = ff_to_double_fast(y);
    const double dot = fma(z, uj.z - ui.z, fma(yy, uj.y - ui.y, x * (uj.x - ui.x)));
    return re * (ry * ry * ry) * dot;
}

// Staging of the mixed build's row outputs: each thread appends the entries of its PPE row
// (column, FP32 coefficient, low part) and of its gradient row to a ring of 12 in shared
// memory (an unconditional store and a cursor step, no branch) and writes each completed
// group of 8 as whole 32-byte sectors (the grouped row layout, sell8), so that no partially
// written sector has to be filled from DRAM.  A check every 2 iterations writes at most one
// completed group per list, which leaves at most 7 unwritten; the next 2 iterations add at
// most 4, so 12 slots never wrap onto an unwritten entry (and 24 KB per 128 threads keeps 8
// blocks on an SM).  Entry-major: thread t's entry e sits at [e][t], consecutive threads in
// consecutive banks.
constexpr int kRing = 16;
// the ring in the block's dynamic shared memory: four arrays of kRing x (block size) words
struct RowStage {
    int32_t* c;
    float* h;
    float* l;
    int32_t* nc;
    int bt;
    __device__ int32_t* col(int e) const { return c + e * bt; }
    __device__ float* hi(int e) const { return h + e * bt; }
    __device__ float* lo(int e) const { return l + e * bt; }
    __device__ int32_t* ncol(int e) const { return nc + e * bt; }
};
// dynamic shared memory of the ring for a block of bt threads (64 KB at 256 threads)
constexpr size_t ring_bytes(int bt) { return 4 * kRing * (size_t)bt * sizeof(int32_t); }

// Entry flags while a PPE row is being assembled (slots are < 2^30)
constexpr int kEntryN = 1 << 30;   // within re_n: contributes to n*
constexpr int kEntryL = 1 << 29;   // non-dummy within re_lap: a PPE coefficient
constexpr int kSlotMask = kEntryL - 1;

// Mixed precision with the PPE: one walk per row over the candidate list, two candidates at
// a time in packed float-float: the squared distance decides membership (float-float
// outside a band of its error around re^2, binary64 inside it), n* and the diagonal are
// accumulated and the PPE coefficients and gradient neighbours written in candidate order.
// Nine in ten candidates are members, so evaluating every candidate wastes little.  With
// the equation of state only the number-density neighbours (one in seven) are members: the
// members are classified and staged first, as on the FP64 path, and only they evaluated.
// FP64: two passes.  Classification decides the predicates (FP32 / float-float / binary64
// tiers) and writes the hits into the row's PPE slots in candidate order (band pairs,
// decided after the walk, last); the dense pass evaluates every hit with (nearly) all
// lanes busy and compacts the PPE coefficients in place to the front of the row.
// Registers: the default mixed and the FP64 instantiations fit 64 (2048 threads per SM);
// the options and the ensemble's take up to 85 (1536).
// KERN, SRC: the weight (0 Eq. 4, 1 cubic) and the PPE source (0 Eq. 13, 1 HS, 2 HS + ECS) as
// compile-time choices, so that the default instantiation carries none of the options' code
template <bool MIXED, int KERN, int SRC, bool MULTI>
__global__ void __launch_bounds__(kBuildBT, (!MULTI && (!MIXED || (KERN == 0 && SRC == 0))) ? 4 : 3)
    k_build(BuildArgs a) {
    // FLUID and WALL rows only (the bucket build's list of them): a DUMMY particle's own n*
    // enters no equation (no free-surface test, no PPE row, no gradient), so it is not
    // evaluated (reported as 0)
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = tid < (int)*a.nrows ? a.rows[tid] : -1;
    // mixed with the PPE: the row-output ring (ring_bytes(blockDim.x) of dynamic shared
    // memory; other launches pass none and never touch it)
    extern __shared__ __align__(16) int32_t s_ring[];
    const int rbt = (int)blockDim.x;
    const RowStage stage{s_ring, (float*)(s_ring + kRing * rbt), (float*)(s_ring + 2 * kRing * rbt),
                         s_ring + 3 * kRing * rbt, rbt};
    bool surf = false, ppe = false;
    unsigned n_lap = 0, n_pnd = 0;   // pairs evaluated by this row
    unsigned n_cand = 0;             // candidate-list entries it classified
    if (i >= 0) {
        Radius rn = a.rn, rl = a.rl;
        double coef_ppe = a.coef_ppe, coef0 = a.coef0, n0 = a.n0;
        ff cre_ff = a.cre_ff, ncoef_ff = a.ncoef_ff;
        if (MULTI) {   // the row's scene
            const SceneParams& sp = a.scn[a.sid[i]];
            rn = sp.rn;
            rl = sp.rl;
            coef_ppe = sp.coef_ppe;
            coef0 = sp.coef_lap;
            n0 = sp.n0_pnd;
            cre_ff = a.rho_s ? ff{sp.cre2_h, sp.cre2_l} : ff{sp.cre_h, sp.cre_l};
            ncoef_ff = a.rho_s ? ff{sp.ncoef2_h, sp.ncoef2_l} : ff{sp.ncoef_h, sp.ncoef_l};
        }
        const float4 ih = a.pos32[i], il = a.pff[2 * i + 1];
        const double4 pi = a.pos[i];
        const int cnt = a.vcnt[i];
        const bool with_ppe = (a.pressure_mode == 0);
        int m_f = 0, out_n = 0, m_n = 0;   // m_n: entries within re_n (number density)
        bool overflow = false;
        // a decided pair: into the gradient list and the row's PPE slots
        auto append = [&](int j, bool tl, bool tn, bool nb_ok) {
            if (!tl && !tn) return;
            if (tn && nb_ok) {
                if (out_n < a.cap_n) a.n_col[sell8(i, out_n, a.cap_n)] = j;
                out_n++;
            }
            if (m_f >= a.cap) {
                overflow = true;
                return;
            }
            // every hit in candidate order: the rows of a slice (neighbouring particles, one
            // candidate sequence) then hold nearby particles at the same entry, which keeps
            // the solver's gathers of x[col] within few cache lines per warp
            a.lap_col[sell8(i, m_f++, a.cap)] = j | (tn ? kEntryN : 0) | (tl ? kEntryL : 0);
            m_n += tn ? 1 : 0;
        };
        // FP64 path: classification first (the mixed path decides membership inside its
        // single walk below).  Band pairs are set aside and decided after the walk, so that
        // the lanes of a warp take the float-float and binary64 tiers together
        if (!MIXED || !with_ppe) {
        constexpr int kPend = 16;
        int pend[kPend];
        int np = 0;
        // ---- classification
        int jn = cnt > 1 ? a.vcol[sell8(i, 1, a.cap_v)] : 0;
        int j0 = cnt > 0 ? a.vcol[sell8(i, 0, a.cap_v)] : 0;
        float4 qn = a.pos32[j0];
        for (int k = 0; k < cnt; k++) {
            const int j = j0;
            const float4 jh = qn;
            j0 = jn;
            if (k + 1 < cnt) qn = a.pos32[jn];
            if (k + 2 < cnt) jn = a.vcol[sell8(i, k + 2, a.cap_v)];
            const float r2 = dist2_f(ih, jh);
            const bool nb_ok = kind_of(jh) != kDummy;
            int tl = (nb_ok && with_ppe) ? tier1(r2, rl) : 0;
            int tn = tier1(r2, rn);
            if (!tl && !tn) continue;
            if (tl == 2 || tn == 2) {
                if (np < kPend) {
                    pend[np++] = k;
                    continue;
                }
                const ff r2f = pair_r2(ih, il, jh, a.pff[2 * j + 1]);
                if (tl == 2) tl = decide_band(r2f, rl, a.pos, pi, j) ? 1 : 0;
                if (tn == 2) tn = decide_band(r2f, rn, a.pos, pi, j) ? 1 : 0;
            }
            append(j, tl, tn, nb_ok);
        }
        for (int q = 0; q < np; q++) {
            const int j = a.vcol[sell8(i, pend[q], a.cap_v)];
            const float4 jh = a.pos32[j];
            const float r2 = dist2_f(ih, jh);
            const bool nb_ok = kind_of(jh) != kDummy;
            int tl = (nb_ok && with_ppe) ? tier1(r2, rl) : 0;
            int tn = tier1(r2, rn);
            const ff r2f = pair_r2(ih, il, jh, a.pff[2 * j + 1]);
            if (tl == 2) tl = decide_band(r2f, rl, a.pos, pi, j) ? 1 : 0;
            if (tn == 2) tn = decide_band(r2f, rn, a.pos, pi, j) ? 1 : 0;
            append(j, tl, tn, nb_ok);
        }
        }
        // ---- dense evaluation and in-place compaction (write slot <= read slot)
        double nd = 0.0, dg = 0.0, hs = 0.0;   // hs: sum of the HS source terms
        int out_l = 0;
        const int m_all = m_f;
        auto slot_of = [&](int t) { return t; };
        if constexpr (MIXED) {
            // Two entries per iteration, their pair terms in packed FP32x2 float-float.
            // 1/r: one Newton step (~1e-13) serves the PPE coefficient; n* takes a second
            // (~1e-15) so that it stays far inside the flag band.  The terms are summed in
            // entry order into (n*, diagonal) as one packed float-float accumulator; an
            // entry without a term adds an exact zero.
            ff2 acc = {f2(0.f), f2(0.f)};
            const ff2 ren = {f2(rn.re_f), f2(rn.re_l)};
            const ff2 cre = {f2(cre_ff.h), f2(cre_ff.l)};
            const ff2 ncoef = {f2(ncoef_ff.h), f2(ncoef_ff.l)};
            const float2 rhoi = a.rho_ff ? a.rho_ff[i] : make_float2(0.f, 0.f);
            const ff2 coef = {f2(-ncoef_ff.h), f2(-ncoef_ff.l)};
            const ff2 invn = {f2(rn.inv_f), f2(rn.inv_l)}, invl = {f2(rl.inv_f), f2(rl.inv_l)};
            const double4 ui = SRC >= 1 ? a.vel_star[i] : make_double4(0.0, 0.0, 0.0, 0.0);
            // the row's outputs, staged 8 entries at a time (RowStage above)
            const int t_ = threadIdx.x;
            // group g of a list sits in ring half g & 1
            auto flush_lap = [&](int g) {
                const size_t q = sell8(i, 8 * g, a.cap);
                const int h = (g & 1) * 8;
                *(int4*)(a.lap_col + q) = make_int4(stage.col(h)[t_], stage.col(h + 1)[t_],
                                                    stage.col(h + 2)[t_], stage.col(h + 3)[t_]);
                *(int4*)(a.lap_col + q + 4) = make_int4(stage.col(h + 4)[t_], stage.col(h + 5)[t_],
                                                        stage.col(h + 6)[t_], stage.col(h + 7)[t_]);
                *(float4*)(a.lap_v32 + q) = make_float4(stage.hi(h)[t_], stage.hi(h + 1)[t_],
                                                        stage.hi(h + 2)[t_], stage.hi(h + 3)[t_]);
                *(float4*)(a.lap_v32 + q + 4) = make_float4(stage.hi(h + 4)[t_], stage.hi(h + 5)[t_],
                                                            stage.hi(h + 6)[t_], stage.hi(h + 7)[t_]);
                *(float4*)(a.lap_vlo + q) = make_float4(stage.lo(h)[t_], stage.lo(h + 1)[t_],
                                                        stage.lo(h + 2)[t_], stage.lo(h + 3)[t_]);
                *(float4*)(a.lap_vlo + q + 4) = make_float4(stage.lo(h + 4)[t_], stage.lo(h + 5)[t_],
                                                            stage.lo(h + 6)[t_], stage.lo(h + 7)[t_]);
            };
            auto flush_n = [&](int g) {
                const size_t q = sell8(i, 8 * g, a.cap_n);
                const int h = (g & 1) * 8;
                *(int4*)(a.n_col + q) = make_int4(stage.ncol(h)[t_], stage.ncol(h + 1)[t_],
                                                  stage.ncol(h + 2)[t_], stage.ncol(h + 3)[t_]);
                *(int4*)(a.n_col + q + 4) = make_int4(stage.ncol(h + 4)[t_], stage.ncol(h + 5)[t_],
                                                      stage.ncol(h + 6)[t_], stage.ncol(h + 7)[t_]);
            };
            auto put_lap = [&](int j, float h, float l, bool on) {
                const int e = out_l & (kRing - 1);
                stage.col(e)[t_] = j;
                stage.hi(e)[t_] = h;
                stage.lo(e)[t_] = l;
                out_l += on ? 1 : 0;
            };
            auto put_n = [&](int j, bool on) {
                stage.ncol(out_n & (kRing - 1))[t_] = j;
                out_n += on ? 1 : 0;
            };
            int done_l = 0, done_n = 0;   // groups written
            auto flush_ready = [&]() {
                const bool fl = done_l < (min(out_l, a.cap) >> 3);
                const bool fn = done_n < (min(out_n, a.cap_n) >> 3);
                if (__any_sync(__activemask(), fl || fn)) {
                    if (fl) flush_lap(done_l++);
                    if (fn) flush_n(done_n++);
                }
            };
            // the members' terms of a pair of candidates (lane x: j0, lane y: j1), shared by
            // the single walk and the walk over staged entries
            auto terms = [&](int j0, int j1, const ff2& dx, const ff2& dy, const ff2& dz,
                             const ff2& r2, bool tn0, bool tl0, bool tn1, bool tl1) {
                const ff2 y = ff2_rsqrt1(r2);
                // the number-density weight of both lanes, used only where tn (a branch on
                // tn0 || tn1 would be taken by nearly every warp anyway)
                const ff2 y2 = ff2_rsqrt_step(r2, y);
                const ff2 w = KERN == 1 ? ff2_cube(ff2_one_minus(ff2_mul(ff2_mul(r2, y2), invn)))
                                        : ff2_mul_add(ren, y2, {f2(-1.f), f2(0.f)});
                if (SRC >= 1) {
                    // HS: re_n / r^3 (r_ij . (u*_j - u*_i)), binary64 from the float-float
                    // offsets and reciprocal distance
                    if (tn0) hs += hs_term(ff2_lo(dx), ff2_lo(dy), ff2_lo(dz), ff2_lo(y2),
                                           a.vel_star[j0], ui, rn.re);
                    if (tn1) hs += hs_term(ff2_hi(dx), ff2_hi(dy), ff2_hi(dz), ff2_hi(y2),
                                           a.vel_star[j1], ui, rn.re);
                }
                // c = coef (re/r - 1) = (coef re) y - coef, or coef (1 - r/re)^3
                ff2 c = KERN == 1 ? ff2_mul(coef, ff2_cube(ff2_one_minus(ff2_mul(ff2_mul(r2, y), invl))))
                                      : ff2_mul_add(cre, y, ncoef);
                if (a.rho_ff) {   // two-phase: times 2/(rho_i + rho_j)
                    const float2 q0 = a.rho_ff[j0], q1 = a.rho_ff[j1];
                    c = ff2_mul(c, ff2_two_over(ff2_add({f2(rhoi.x), f2(rhoi.y)},
                                                        {make_float2(q0.x, q1.x), make_float2(q0.y, q1.y)})));
                }
                acc = ff2_add(acc, {make_float2(tn0 ? w.h.x : 0.f, tl0 ? c.h.x : 0.f),
                                    make_float2(tn0 ? w.l.x : 0.f, tl0 ? c.l.x : 0.f)});
                acc = ff2_add(acc, {make_float2(tn1 ? w.h.y : 0.f, tl1 ? c.h.y : 0.f),
                                    make_float2(tn1 ? w.l.y : 0.f, tl1 ? c.l.y : 0.f)});
                if (with_ppe) {   // the ring exists only in the PPE launch (block-uniform)
                    put_lap(j0, c.h.x, c.l.x, tl0);
                    put_lap(j1, c.h.y, c.l.y, tl1);
                }
            };
            if (!with_ppe) {
                // equation of state: one in seven candidates is a member (within re_n), so
                // the classification above staged the members and only they are evaluated
                for (int t = 0; t < m_all; t += 2) {
                    const bool two = t + 1 < m_all;
                    const int e0 = a.lap_col[sell8(i, t, a.cap)];
                    const int e1 = two ? a.lap_col[sell8(i, t + 1, a.cap)] : e0;
                    const int j0 = e0 & kSlotMask, j1 = e1 & kSlotMask;
                    const float4 h0 = a.pff[2 * j0], l0 = a.pff[2 * j0 + 1];
                    const float4 h1 = a.pff[2 * j1], l1 = a.pff[2 * j1 + 1];
                    const ff2 dx = ff2_diff(ih.x, il.x, make_float2(h0.x, h1.x), make_float2(l0.x, l1.x));
                    const ff2 dy = ff2_diff(ih.y, il.y, make_float2(h0.y, h1.y), make_float2(l0.y, l1.y));
                    const ff2 dz = ff2_diff(ih.z, il.z, make_float2(h0.z, h1.z), make_float2(l0.z, l1.z));
                    const ff2 r2 = ff2_dist2(dx, dy, dz);
                    const bool ok0 = r2.h.x > 0.f, ok1 = two && r2.h.y > 0.f;
                    if (!ok0 && !(exact_dist2(pi, a.pos[j0]) > 0.0)) atomicOr(&a.st->err, kErrCoincident);
                    if (two && !ok1 && !(exact_dist2(pi, a.pos[j1]) > 0.0))
                        atomicOr(&a.st->err, kErrCoincident);
                    terms(j0, j1, dx, dy, dz, r2, ok0 && (e0 & kEntryN), false,
                          ok1 && (e1 & kEntryN), false);
                }
            } else {
                // One walk over the candidate list, two candidates per iteration: the float-float
                // squared distance decides membership (the second tier of the exact predicate:
                // outside the ff_tol band around re^2, binary64 inside it) and the members' terms
                // are evaluated at once, in candidate order.  The slots of the next pair are
                // loaded one iteration ahead.
                int s0 = cnt > 0 ? a.vcol[sell8(i, 0, a.cap_v)] : 0;
                int s1 = cnt > 1 ? a.vcol[sell8(i, 1, a.cap_v)] : s0;
                for (int t = 0; t < cnt; t += 2) {
                    const bool two = t + 1 < cnt;
                    const int j0 = s0, j1 = s1;
                    if (t + 2 < cnt) {
                        s0 = a.vcol[sell8(i, t + 2, a.cap_v)];
                        s1 = t + 3 < cnt ? a.vcol[sell8(i, t + 3, a.cap_v)] : s0;
                    }
                    const float4 h0 = a.pff[2 * j0], l0 = a.pff[2 * j0 + 1];
                    const float4 h1 = a.pff[2 * j1], l1 = a.pff[2 * j1 + 1];
                    const ff2 dx = ff2_diff(ih.x, il.x, make_float2(h0.x, h1.x), make_float2(l0.x, l1.x));
                    const ff2 dy = ff2_diff(ih.y, il.y, make_float2(h0.y, h1.y), make_float2(l0.y, l1.y));
                    const ff2 dz = ff2_diff(ih.z, il.z, make_float2(h0.z, h1.z), make_float2(l0.z, l1.z));
                    const ff2 r2 = ff2_dist2(dx, dy, dz);
                    // membership: d = r^2 - re^2 in float-float, decided outside [-ff_tol, ff_tol];
                    // inside that band binary64 decides, in a branch the warp enters only when
                    // one of its lanes has such a pair (rare)
                    const float2 dn = add2(sub2(r2.h, f2(rn.re2_h)), sub2(r2.l, f2(rn.re2_l)));
                    const float2 dl = add2(sub2(r2.h, f2(rl.re2_h)), sub2(r2.l, f2(rl.re2_l)));
                    const bool nb0 = kind_of(h0) != kDummy, nb1 = kind_of(h1) != kDummy;
                    bool tn0 = dn.x <= -rn.ff_tol, tn1 = two && dn.y <= -rn.ff_tol;
                    bool tl0 = nb0 && dl.x <= -rl.ff_tol, tl1 = two && nb1 && dl.y <= -rl.ff_tol;
                    const bool bn0 = !(dn.x <= -rn.ff_tol) && dn.x < rn.ff_tol;
                    const bool bn1 = two && !(dn.y <= -rn.ff_tol) && dn.y < rn.ff_tol;
                    const bool bl0 = nb0 && !(dl.x <= -rl.ff_tol) && dl.x < rl.ff_tol;
                    const bool bl1 = two && nb1 && !(dl.y <= -rl.ff_tol) && dl.y < rl.ff_tol;
                    if (__any_sync(__activemask(), bn0 || bn1 || bl0 || bl1)) {
                        if (bn0 || bl0) {
                            const double d2 = exact_dist2(pi, a.pos[j0]);
                            if (bn0) tn0 = d2 < rn.re2;
                            if (bl0) tl0 = d2 < rl.re2;
                        }
                        if (bn1 || bl1) {
                            const double d2 = exact_dist2(pi, a.pos[j1]);
                            if (bn1) tn1 = d2 < rn.re2;
                            if (bl1) tl1 = d2 < rl.re2;
                        }
                    }
                    // a member at zero distance (coincident to float-float) is an error unless
                    // binary64 separates it; either way it adds no term
                    const bool ok0 = r2.h.x > 0.f, ok1 = two && r2.h.y > 0.f;
                    const bool z0 = (tn0 || tl0) && !ok0, z1 = (tn1 || tl1) && !ok1;
                    if (__any_sync(__activemask(), z0 || z1)) {
                        if (z0 && !(exact_dist2(pi, a.pos[j0]) > 0.0)) atomicOr(&a.st->err, kErrCoincident);
                        if (z1 && !(exact_dist2(pi, a.pos[j1]) > 0.0)) atomicOr(&a.st->err, kErrCoincident);
                    }
                    // the gradient list: non-dummy members within re_n, in candidate order
                    put_n(j0, tn0 && nb0);
                    put_n(j1, tn1 && nb1);
                    m_n += (tn0 ? 1 : 0) + (tn1 ? 1 : 0);
                    tn0 = tn0 && ok0;
                    tn1 = tn1 && ok1;
                    tl0 = tl0 && ok0;
                    tl1 = tl1 && ok1;
                    terms(j0, j1, dx, dy, dz, r2, tn0, tl0, tn1, tl1);
                    if ((t & 6) == 6) flush_ready();   // every 4 iterations
                }
                flush_ready();   // the last completed groups (at most one per list)
                if (out_l > a.cap) {
                    overflow = true;
                    out_l = a.cap;
                }
                // the last, partial groups: the PPE row padded with zero coefficients on the
                // row's own column (the solver reads whole groups), the gradient row as is
                if (out_l & 7) {
                    const int h = ((out_l >> 3) & 1) * 8;
                    for (int e = out_l & 7; e < 8; e++) {
                        stage.col(h + e)[t_] = i;
                        stage.hi(h + e)[t_] = 0.f;
                        stage.lo(h + e)[t_] = 0.f;
                    }
                    flush_lap(out_l >> 3);
                }
                const int mn = min(out_n, a.cap_n);
                if (mn & 7) {
                    const int h = ((mn >> 3) & 1) * 8;
                    for (int e = mn & 7; e < 8; e++) stage.ncol(h + e)[t_] = i;
                    flush_n(mn >> 3);
                }
            }
            nd = ff_to_double_fast(ff2_lo(acc));
            dg = ff_to_double_fast(ff2_hi(acc));
        } else {
            for (int t = 0; t < m_all; t++) {
                const int e = a.lap_col[sell8(i, slot_of(t), a.cap)];
                const int j = e & kSlotMask;
                const bool tn = (e & kEntryN) != 0, tl = (e & kEntryL) != 0;
                const double4 pj = a.pos[j];
                const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                const double rr2 = fma(dz, dz, fma(dy, dy, dx * dx));
                if (!(rr2 > 0.0)) {
                    atomicOr(&a.st->err, kErrCoincident);
                    continue;
                }
                const double rs = rsqrt(rr2);
                if (tn) {
                    nd += KERN == 1 ? cubic_w_d(rr2, rs, rn.inv_re) : fma(rn.re, rs, -1.0);
                    if (SRC >= 1) {
                        const double4 uj = a.vel_star[j], ui = a.vel_star[i];
                        const double dot = fma(dz, uj.z - ui.z, fma(dy, uj.y - ui.y, dx * (uj.x - ui.x)));
                        hs += rn.re * (rs * rs * rs) * dot;
                    }
                }
                if (tl) {
                    const double wl = KERN == 1 ? cubic_w_d(rr2, rs, rl.inv_re) : fma(rl.re, rs, -1.0);
                    const double cd =
                        a.rho_s ? (coef0 * (2.0 / (a.rho_s[i] + a.rho_s[j]))) * wl : coef_ppe * wl;
                    dg += cd;
                    const size_t q = sell8(i, out_l++, a.cap);
                    a.lap_col[q] = j;
                    a.lap_v64[q] = cd;
                }
            }
        }
        surf = nd < a.beta * n0;
        ppe = !surf;
        a.nstar[i] = nd;
        a.flag[i] = surf ? 1 : 0;
        if (!ppe) a.bvec[i] = 0.0;
        else if (SRC >= 1) {
            double bv = -hs / (n0 * a.dt);   // (Dn/Dt)* / (n0 dt)
            if (SRC == 2) {                    // + ECS / dt (Eq. 24-25)
                const double dk = a.ecs_dk[i], eps = (a.ecs_nk[i] - n0) / n0;
                const double ecs = fabs(eps) * (dk / n0) + fabs(a.dt * dk / n0) * (eps / a.dt);
                bv += ecs / a.dt;
            }
            a.bvec[i] = bv;
        }
        else a.bvec[i] = a.inv_dt2 * ((nd - n0) / n0);
        const double dgv = ppe ? dg + a.diag_add : 0.0;
        a.diag[i] = dgv;
        a.diag32[i] = (float)dgv;
        a.lap_cnt[i] = out_l;
        a.n_cnt[i] = min(out_n, a.cap_n);
        if (overflow || out_n > a.cap_n) atomicOr(&a.st->err, kErrCap);
        if (a.pressure_mode == 1) {
            const double k = a.rho_s ? a.rho_s[i] * a.wc_c : a.wc_k;   // rho_i c0^2 / gamma
            a.p[i] = ppe ? k * (pow(nd / n0, a.gamma) - 1.0) : 0.0;
        }
        n_lap = (unsigned)out_l;
        n_pnd = (unsigned)m_n;
        n_cand = (unsigned)cnt;
    }
    const unsigned bs = __ballot_sync(0xffffffffu, surf), bp = __ballot_sync(0xffffffffu, ppe);
    for (int o = 16; o > 0; o >>= 1) {
        n_lap += __shfl_xor_sync(0xffffffffu, n_lap, o);
        n_pnd += __shfl_xor_sync(0xffffffffu, n_pnd, o);
        n_cand += __shfl_xor_sync(0xffffffffu, n_cand, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_cand) atomicAdd(&a.st->list_tests, (unsigned long long)n_cand);
        if (bs) atomicAdd(&a.st->n_surface, (unsigned)__popc(bs));
        if (bp) atomicAdd(&a.st->n_ppe, (unsigned)__popc(bp));
        if (n_lap) atomicAdd(&a.st->pairs_lap, (unsigned long long)n_lap);
        if (n_pnd) atomicAdd(&a.st->pairs_n, (unsigned long long)n_pnd);
    }
}
// ---------------------------------------------------------------- ECS rates at r^k
// The error-compensating source (Eq. 24) needs, per FLUID / WALL row, the number density
// n^k and its rate (Dn/Dt)^k = -sum re_n/r^3 (r_ij . u_ij) at the step's start r^k, u^k,
// over the number-density neighbours (re_n, every non-GHOST kind; the exact predicate as
// in the build).  Mixed mode: float-float distances, binary64 rate terms.
struct RatesArgs {
    int cap_v;
    const int32_t* vcol;
    const int32_t* vcnt;
    const float4* pos32;
    const float4* pos32lo;
    const double4* pos;
    const double4* vel;
    const int32_t* rows;
    const uint32_t* nrows;
    Radius rn;
    double* nk;
    double* dk;
    const uint16_t* sid;
    const SceneParams* scn;
};

template <bool MIXED>
__global__ void __launch_bounds__(kBT) k_ecs_rates(RatesArgs a) {
    const int tid = blockIdx.x * kBT + threadIdx.x;
    if (tid >= (int)*a.nrows) return;
    const int i = a.rows[tid];
    const Radius rn = a.sid ? a.scn[a.sid[i]].rn : a.rn;
    const float4 ih = a.pos32[i], il = a.pos32lo[i];
    const double4 pi = a.pos[i], ui = a.vel[i];
    const int cnt = a.vcnt[i];
    ff nf = {0.f, 0.f};
    double nd = 0.0, dd = 0.0;
    for (int k = 0; k < cnt; k++) {
        const int j = a.vcol[sell8(i, k, a.cap_v)];
        const float4 jh = a.pos32[j];
        const float r2 = dist2_f(ih, jh);
        int t = tier1(r2, rn);
        if (!t) continue;
        const float4 jl = a.pos32lo[j];
        if (t == 2 && !decide_band(pair_r2(ih, il, jh, jl), rn, a.pos, pi, j)) continue;
        const double4 uj = a.vel[j];
        if (MIXED) {
            const ff dx = ff_diff(ih.x, il.x, jh.x, jl.x), dy = ff_diff(ih.y, il.y, jh.y, jl.y);
            const ff dz = ff_diff(ih.z, il.z, jh.z, jl.z);
            const ff rr = ff_dist2(dx, dy, dz);
            if (!(rr.h > 0.f)) continue;   // coincident pairs are reported by the prediction
            const ff y = ff_rsqrt(rr);
            nf = ff_add(nf, ff_add_f(ff_mul({rn.re_f, rn.re_l}, y), -1.f));
            dd += hs_term(dx, dy, dz, y, uj, ui, rn.re);
        } else {
            const double4 pj = a.pos[j];
            const double dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
            const double rr2 = fma(dz, dz, fma(dy, dy, dx * dx));
            if (!(rr2 > 0.0)) continue;
            const double rs = rsqrt(rr2);
            nd += fma(rn.re, rs, -1.0);
            const double dot = fma(dz, uj.z - ui.z, fma(dy, uj.y - ui.y, dx * (uj.x - ui.x)));
            dd += rn.re * (rs * rs * rs) * dot;
        }
    }
    a.nk[i] = MIXED ? ff_to_double_fast(nf) : nd;
    a.dk[i] = -dd;
}
}  // namespace

void launch_ecs_rates(Ctx* c) {
    RatesArgs a;
    a.cap_v = c->cap_v;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.pos32 = c->pos32;
    a.pos32lo = c->pos32lo;
    a.pos = c->pos;
    a.vel = c->vel;
    a.rows = c->rows_fw;
    a.nrows = c->scan_fw + c->n;
    a.rn = c->r_n;
    a.nk = c->ecs_nk;
    a.dk = c->ecs_dk;
    a.sid = c->sid;
    a.scn = c->scn;
    const int grid = (int)((c->n + kBT - 1) / kBT);
    if (c->prm.precision == 1) k_ecs_rates<true><<<grid, kBT, 0, c->stream>>>(a);
    else k_ecs_rates<false><<<grid, kBT, 0, c->stream>>>(a);
    c->launches += 1;
}

// threads per row of the prediction (tuned: 1, 2 or 4)
template <bool MIXED, bool MULTI>
static void predict_tpr(Ctx* c, const PredictArgs& a) {
    const int tpr = c->predict_tpr;
    const int grid = (int)(((int64_t)c->n * tpr + kBT - 1) / kBT);
    if (tpr == 4) k_predict<MIXED, MULTI, 4><<<grid, kBT, 0, c->stream>>>(a);
    else if (tpr == 2) k_predict<MIXED, MULTI, 2><<<grid, kBT, 0, c->stream>>>(a);
    else k_predict<MIXED, MULTI, 1><<<grid, kBT, 0, c->stream>>>(a);
}

void launch_predict_rows(Ctx* c) {
    const mps_params& P = c->prm;
    PredictArgs a;
    a.n = (int)c->n;
    a.cap_v = c->cap_v;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.pos32 = c->pos32;
    a.pos32lo = c->pos32lo;
    a.pos = c->pos;
    a.pos_b = c->pos_b;
    a.rows = c->rows_f;
    a.nrows = c->scan_f + c->n;
    a.nu_s = c->nu_s;
    a.kernel = P.kernel;   // predict
    a.vel = c->vel;
    a.vel32 = c->vel32;
    a.type = c->type;
    a.pos_star = c->pos_star;
    a.vel_star = c->vel_star;
    a.pos32_star = c->pos32_star;
    a.pff_star = c->pff_star;
    a.st = c->st;
    a.r = c->r_lap;
    a.coef_lap = c->coef_lap;
    a.nu = P.nu;
    a.dt = P.dt;
    a.g0 = P.g[0];
    a.g1 = P.g[1];
    a.g2 = c->dim == 3 ? P.g[2] : 0.0;
    a.g_dev = c->capture_ctl ? c->capture_ctl->g : nullptr;
    a.bmin0 = c->grid.bmin[0];
    a.bmin1 = c->grid.bmin[1];
    a.bmin2 = c->grid.bmin[2];
    a.sid = c->sid;
    a.scn = c->scn;
    const bool multi = c->n_scenes > 1;
    if (P.precision == 1) {
        if (multi) predict_tpr<true, true>(c, a);
        else predict_tpr<true, false>(c, a);
    } else {
        if (multi) predict_tpr<false, true>(c, a);
        else predict_tpr<false, false>(c, a);
    }
    c->launches += 1;
}

// (kernel, source): (0, 0), (0, 1), (0, 2), (1, 0); the cubic weight with HS is rejected
template <bool MULTI>
static int allow_ring_t(Ctx* c) {
    // the ring of a 256-thread block (64 KB) is above the default 48 KB of dynamic shared
    // memory of a launch
    const int b = (int)ring_bytes(256);
    MPS_CUDA(c, cudaFuncSetAttribute(k_build<true, 1, 0, MULTI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    MPS_CUDA(c, cudaFuncSetAttribute(k_build<true, 0, 0, MULTI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    MPS_CUDA(c, cudaFuncSetAttribute(k_build<true, 0, 1, MULTI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    MPS_CUDA(c, cudaFuncSetAttribute(k_build<true, 0, 2, MULTI>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, b));
    return MPS_OK;
}

template <bool MULTI>
static void launch_build_t(Ctx* c, const BuildArgs& a) {
    const mps_params& P = c->prm;
    // the source term enters the PPE only: an equation-of-state step takes the standard one
    // (the ECS rates are not even allocated then)
    const int src = P.pressure_mode == 0 ? P.source_term : 0;
    const bool ring = P.precision == 1 && P.pressure_mode == 0;
    const int bt = build_block_of(c);
    const size_t sm = ring ? ring_bytes(bt) : 0;
    const int grid = (int)((c->n + bt - 1) / bt);
    if (P.precision == 1) {
        if (P.kernel == 1) k_build<true, 1, 0, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else if (src == 0) k_build<true, 0, 0, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else if (src == 1) k_build<true, 0, 1, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else k_build<true, 0, 2, MULTI><<<grid, bt, sm, c->stream>>>(a);
    } else {
        if (P.kernel == 1) k_build<false, 1, 0, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else if (src == 0) k_build<false, 0, 0, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else if (src == 1) k_build<false, 0, 1, MULTI><<<grid, bt, sm, c->stream>>>(a);
        else k_build<false, 0, 2, MULTI><<<grid, bt, sm, c->stream>>>(a);
    }
}

__global__ void __launch_bounds__(kBT)
    k_clear_rows(int n, double* nstar, uint8_t* flag, double* diag, float* diag32, double* bvec,
                 int32_t* lap_cnt, int32_t* n_cnt, double* p) {
    const int i = blockIdx.x * kBT + threadIdx.x;
    if (i >= n) return;
    nstar[i] = 0.0;
    flag[i] = 0;
    diag[i] = 0.0;
    diag32[i] = 0.f;
    bvec[i] = 0.0;
    lap_cnt[i] = 0;
    n_cnt[i] = 0;
    if (p) p[i] = 0.0;
}

void launch_clear_rows(Ctx* c) {
    const int n = (int)c->n;
    k_clear_rows<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(
        n, c->nstar, c->flag, c->diag, c->diag32, c->bvec, c->nb_lap_cnt, c->nb_n_cnt,
        c->prm.pressure_mode == 1 ? c->p : nullptr);
    c->launches += 1;
}

int build_block_of(const Ctx* c) {
    if (c->build_block) return c->build_block;
    return (c->prm.precision == 1 && c->prm.pressure_mode == 0) ? kBuildRingBT : kBuildBT;
}

int build_rows_init(Ctx* c) {
    int rc = allow_ring_t<false>(c);
    return rc ? rc : allow_ring_t<true>(c);
}

void launch_build_rows(Ctx* c) {
    const mps_params& P = c->prm;
    BuildArgs a;
    a.n = (int)c->n;
    a.cap_v = c->cap_v;
    a.cap = c->cap;
    a.cap_n = c->cap_n;
    a.pressure_mode = P.pressure_mode;
    a.rows = c->rows_fw;
    a.nrows = c->scan_fw + c->n;
    a.rho_s = c->rho_s;
    a.rho_ff = c->rho_ff;
    a.coef0 = c->coef_lap;   // 2d/(n0_lap lambda), the Laplacian's coefficient
    a.kernel = P.kernel;
    a.source = P.source_term;
    a.vel_star = c->vel_star;
    a.dt = P.dt;
    a.ecs_nk = c->ecs_nk;
    a.ecs_dk = c->ecs_dk;
    a.wc_c = P.c0 * P.c0 / P.gamma;
    a.vcol = c->vl_col;
    a.vcnt = c->vl_cnt;
    a.pos32 = c->pos32_star;
    a.pff = c->pff_star;
    a.pos = c->pos_star;
    a.type = c->type;
    a.st = c->st;
    a.rn = c->r_n;
    a.rl = c->r_lap;
    a.coef_ppe = c->coef_ppe;
    // the coefficient without the pair factor when densities are per particle
    const double cpf = c->rho_s ? c->coef_lap : c->coef_ppe;
    a.cre_ff = ff_from_double(cpf * c->r_lap.re);
    a.ncoef_ff = ff_from_double(-cpf);
    a.n0 = c->n0_pnd;
    a.beta = P.beta;
    a.inv_dt2 = c->inv_dt2;
    a.diag_add = c->diag_add;
    a.wc_k = P.rho * P.c0 * P.c0 / P.gamma;
    a.gamma = P.gamma;
    a.lap_col = c->nb_lap_col;
    a.lap_v64 = c->nb_lap_v64;
    a.lap_v32 = c->nb_lap_v32;
    a.lap_vlo = c->nb_lap_vlo;
    a.lap_cnt = c->nb_lap_cnt;
    a.n_col = c->nb_n_col;
    a.n_cnt = c->nb_n_cnt;
    a.nstar = c->nstar;
    a.flag = c->flag;
    a.bvec = c->bvec;
    a.diag = c->diag;
    a.diag32 = c->diag32;
    a.p = c->p;

    a.sid = c->sid;
    a.scn = c->scn;
    if (c->n_scenes > 1) launch_build_t<true>(c, a);
    else launch_build_t<false>(c, a);
    c->launches += 1;
}

}  // namespace mps
