// ppe.cu -- conjugate-gradient solve of the PPE A p = b (Eq. 13 assembled as in the CUDA
// PPE listing (Listing 2) of Sec. 4.3; the paper solves it by (IC)CG, Sec. 3.1.2 and Sec. 4.3).
//
// A is applied from the per-step neighbour lists built at r* (sell8 rows, one thread per
// row; the allocation-free entry point below takes caller rows in plain row-major layout):
//   (A x)_i = diag_i x_i - sum_{j in nb_lap(i)} c_ij x_j   for rows of the PPE (diag_i > 0),
//   (A x)_i = 0 elsewhere,
// where every CG vector vanishes outside the PPE rows, so neighbours j outside them drop out
// of the sum exactly as the off-diagonal entries of the listing do.
//
// FP64 mode: textbook CG in binary64 with stored FP64 coefficients; the recurrence residual
// stops the iteration and the true residual b - A p is recomputed, restarting if needed.
// Mixed mode: outer refinement in binary64 (x and the residual b - A x in binary64, the
// products of A x formed in float-float from float-float coefficients), inner CG in FP32 on
// A e = r/|r| with FP32 coefficients (stored, or recomputed from the FP32 positions:
// matrix-free), FP64 dot products.
//
// Reductions are deterministic: per-block partials summed in block order by the last block.
// Convergence is decided on the device.  The mixed solve (one scene or an ensemble) runs as
// one CUDA graph whose conditional WHILE nodes the kernels drive (build_mixed_graph below);
// the FP64 solve, the adjoint solve and ppe_host_loop = 1 poll one flag per chunk of
// iterations from the host.
#include <cmath>
#include <mutex>

#include "ff.cuh"
#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 256;
constexpr int kWarps = kBT / 32;
// smallest relative reduction asked of one FP32 inner solve (its rounding floor is ~1e-7)
constexpr double kInnerFloor = 1e-6;

// Plain-data view of a row-major PPE operator (the allocation-free entry point's layout).
struct PpeView {
    int n, cap;
    const int32_t* col;
    const int32_t* cnt;
    const double* v64;
    const float* v32;
    const double* diag;
    const double* bvec;
    const float4* pos32s;
    double* partials;
    unsigned int* counter;
};

// ------------------------------------------------------------------ SpMV building blocks
__device__ __forceinline__ double row_dot64(const PpeView& c, int i, const double* x, int lane) {
    const int cnt = c.cnt[i];
    const size_t base = (size_t)i * c.cap;
    double acc = 0.0;
    for (int k = lane; k < cnt; k += 32) acc = fma(c.v64[base + k], x[c.col[base + k]], acc);
    return warp_sum(acc);
}

// ------------------------------------------------------------------ FP64 kernels
// r = b - A x, d = r; rr = r.r.  set_stop: stop2 = tol2 * rr (first call of a solve).
__global__ void __launch_bounds__(kBT) k_resid64(PpeView c, const double* x, double* r, double* d,
                                                 CgScalars* cg, double tol2, int set_stop,
                                                 int set_cg) {
    __shared__ double sm[kWarps];
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * kBT + threadIdx.x) >> 5, nw = (gridDim.x * kBT) >> 5;
    double part = 0.0;
    for (int i = gw; i < c.n; i += nw) {
        const double dg = c.diag[i];
        double ri = 0.0;
        if (dg != 0.0) {
            const double s = row_dot64(c, i, x, lane);
            ri = c.bvec[i] - (dg * x[i] - s);
        }
        if (lane == 0) {
            r[i] = ri;
            if (d) d[i] = ri;
            part += ri * ri;
        }
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, c.partials, &c.counter[0], &tot, sm) && threadIdx.x == 0) {
        cg->rr = tot;
        if (set_stop) cg->stop2 = tol2 * tot;
        if (set_cg) {
            cg->rho = tot;
            cg->rho0 = tot;
            cg->done = (tot <= cg->stop2) ? 1 : 0;
        }
    }
}

// q = A d, alpha = rho / (d.q)
__global__ void __launch_bounds__(kBT) k_spmv64(PpeView c, const double* d, double* q, CgScalars* cg) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[kWarps];
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * kBT + threadIdx.x) >> 5, nw = (gridDim.x * kBT) >> 5;
    double part = 0.0;
    for (int i = gw; i < c.n; i += nw) {
        const double dg = c.diag[i];
        double qi = 0.0;
        if (dg != 0.0) qi = dg * d[i] - row_dot64(c, i, d, lane);
        if (lane == 0) {
            q[i] = qi;
            part += d[i] * qi;
        }
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, c.partials, &c.counter[1], &tot, sm) && threadIdx.x == 0) {
        cg->dq = tot;
        cg->alpha = (tot > 0.0) ? cg->rho / tot : 0.0;
    }
}

// x += alpha d; r -= alpha q; rho' = r.r; beta = rho'/rho; convergence flag
__global__ void __launch_bounds__(kBT) k_xr64(int n, double* x, double* r, const double* d,
                                              const double* q, CgScalars* cg, double* partials,
                                              unsigned int* counter) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[kWarps];
    const double alpha = cg->alpha;
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        x[i] = fma(alpha, d[i], x[i]);
        const double ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        part += ri * ri;
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, partials, counter, &tot, sm) && threadIdx.x == 0) {
        cg->beta = (cg->rho > 0.0) ? tot / cg->rho : 0.0;
        cg->rho = tot;
        cg->iters += 1;
        if (tot <= cg->stop2 || cg->iters >= cg->max_iters || !(cg->dq > 0.0)) cg->done = 1;
    }
}

__global__ void __launch_bounds__(kBT) k_d64(int n, const double* r, double* d, const CgScalars* cg) {
    if (*(volatile const int*)&cg->done) return;
    const double beta = cg->beta;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) d[i] = fma(beta, d[i], r[i]);
}

// ------------------------------------------------------------------ FP32 inner kernels
// r32 = r64 / |r64|, d32 = r32, x32 = 0; rho = r32.r32; stop2 = itol2 * rho.
// itol2 < 0 (the device-driven solve): the inner tolerance and iteration cap are taken on
// the device, as the host loop takes them: the reduction the outer target still needs
// (with a margin of 2) when one FP32 solve can reach it, else inner_tol; h_in (nonzero) is
// the conditional of the inner loop, set to run it unless the inner solve is already done.
__global__ void __launch_bounds__(kBT) k_inner_init(int n, const double* r64, float* r32, float* d32,
                                                    float* x32, CgScalars* cg, double itol2,
                                                    int max_iters, double* partials,
                                                    unsigned int* counter,
                                                    cudaGraphConditionalHandle h_in) {
    __shared__ double sm[kWarps];
    const double scale = 1.0 / sqrt(cg->rr);
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        const float v = (float)(r64[i] * scale);
        r32[i] = v;
        d32[i] = v;
        x32[i] = 0.f;
        part += (double)v * (double)v;
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, partials, counter, &tot, sm) && threadIdx.x == 0) {
        if (itol2 < 0.0) {
            const double need = 0.5 * sqrt(cg->ostop2 / cg->rr);
            const double itol = (need >= kInnerFloor) ? need : cg->inner_tol;
            itol2 = itol * itol;
            max_iters = cg->max_total - cg->total;
        }
        cg->rho = tot;
        cg->rho0 = tot;
        cg->stop2 = itol2 * tot;
        cg->iters = 0;
        cg->max_iters = max_iters;
        cg->done = (tot > 0.0 && max_iters > 0) ? 0 : 1;
        if (h_in) {
            cg->guard_in = 0;
            cudaGraphSetConditional(h_in, cg->done ? 0u : 1u);
        }
    }
}

__global__ void __launch_bounds__(kBT) k_xr32(int n, float* x, float* r, const float* d, const float* q,
                                              CgScalars* cg, double* partials, unsigned int* counter) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[kWarps];
    const float alpha = (float)cg->alpha;
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        x[i] = fmaf(alpha, d[i], x[i]);
        const float ri = fmaf(-alpha, q[i], r[i]);
        r[i] = ri;
        part += (double)ri * (double)ri;
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, partials, counter, &tot, sm) && threadIdx.x == 0) {
        cg->beta = (cg->rho > 0.0) ? tot / cg->rho : 0.0;
        cg->rho = tot;
        cg->iters += 1;
        if (tot <= cg->stop2 || cg->iters >= cg->max_iters || !(cg->dq > 0.0)) cg->done = 1;
    }
}

// d = r + beta d.  h_in (nonzero): the inner loop's conditional, set first by one thread
// (run again unless done; never more than max_total + 2 times in one inner solve)
__global__ void __launch_bounds__(kBT) k_d32(int n, const float* r, float* d, CgScalars* cg,
                                             cudaGraphConditionalHandle h_in) {
    if (h_in && blockIdx.x == 0 && threadIdx.x == 0) {
        const int g = ++cg->guard_in;
        const bool more = !*(volatile const int*)&cg->done && g < cg->max_total + 2;
        cudaGraphSetConditional(h_in, more ? 1u : 0u);
    }
    if (*(volatile const int*)&cg->done) return;
    const float beta = (float)cg->beta;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) d[i] = fmaf(beta, d[i], r[i]);
}

// ------------------------------------------------------------------ thread-per-row (sell8)
// The step's PPE rows are sell8: each thread owns a row, a warp reads a group of 8 entries
// of its 32 rows as 1 KB contiguous, and every FP64 operation runs with all lanes busy.
struct SellView {
    int n, cap;
    const int32_t* col;
    const int32_t* cnt;
    const double* v64;
    const float* v32;
    const float* vlo;
    const double* diag;
    const float* diag32;
    const double* bvec;
    const float4* pos32s;
    double* partials;
    unsigned int* counter;
};

__device__ __forceinline__ double sell_dot64(const SellView& c, int i, const double* x) {
    const int cnt = c.cnt[i];
    double acc = 0.0;
    for (int k = 0; k < cnt; k++) {
        const size_t q = sell8(i, k, c.cap);
        acc = fma(c.v64[q], x[c.col[q]], acc);
    }
    return acc;
}

// sum_k v_k x_{col_k} over one row of the grouped layout (sell8), in entry order: a group's
// 8 columns and 8 coefficients come in as two 16-byte loads each, and the 8 gathers of x
// are issued before their products.  The mixed build pads a row's last group with zero
// coefficients on the row's own column, which add exact zeros.
__device__ __forceinline__ float sell_dot32(const int32_t* __restrict__ cp, const float* __restrict__ vp,
                                            int cnt, const float* __restrict__ x) {
    float acc = 0.f;
    const int ng = (cnt + 7) >> 3;
#pragma unroll 2
    for (int g = 0; g < ng; g++) {
        const int4 c0 = *(const int4*)cp, c1 = *(const int4*)(cp + 4);
        const float4 v0 = *(const float4*)vp, v1 = *(const float4*)(vp + 4);
        const float y0 = x[c0.x], y1 = x[c0.y], y2 = x[c0.z], y3 = x[c0.w];
        const float y4 = x[c1.x], y5 = x[c1.y], y6 = x[c1.z], y7 = x[c1.w];
        acc = fmaf(v0.x, y0, acc);
        acc = fmaf(v0.y, y1, acc);
        acc = fmaf(v0.z, y2, acc);
        acc = fmaf(v0.w, y3, acc);
        acc = fmaf(v1.x, y4, acc);
        acc = fmaf(v1.y, y5, acc);
        acc = fmaf(v1.z, y6, acc);
        acc = fmaf(v1.w, y7, acc);
        cp += 256;
        vp += 256;
    }
    return acc;
}

// r = b - A x, d = r (if d); rr = r.r
__global__ void __launch_bounds__(kBT) k_resid64_t(SellView c, const double* x, double* r,
                                                   double* d, CgScalars* cg, double tol2,
                                                   int set_stop, int set_cg) {
    __shared__ double sm[kWarps];
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < c.n; i += gridDim.x * kBT) {
        const double dg = c.diag[i];
        double ri = 0.0;
        if (dg != 0.0) ri = c.bvec[i] - (dg * x[i] - sell_dot64(c, i, x));
        r[i] = ri;
        if (d) d[i] = ri;
        part = fma(ri, ri, part);
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, c.partials, &c.counter[0], &tot, sm) && threadIdx.x == 0) {
        cg->rr = tot;
        if (set_stop) cg->stop2 = tol2 * tot;
        if (set_cg) {
            cg->rho = tot;
            cg->rho0 = tot;
            cg->done = (tot <= cg->stop2) ? 1 : 0;
        }
    }
}

// mixed outer residual r = b - A x with A's coefficients as float-float (v32 + vlo) and
// x as float-float (xh + xl) beside its binary64 value: each product and the row sum are
// formed with error-free transformations on the FP32 pipes (~2^-46 relative per term), the
// row result is combined with b and the diagonal in binary64.
// h_out (nonzero, the device-driven solve): the sweep's inner iterations are added to the
// total and the refinement loop's conditional is set: another sweep while the residual is
// above the outer target and within the caps (never more than max_outer + 2 sweeps).
template <int BT = kBT>
__global__ void __launch_bounds__(BT) k_resid_ff_t(SellView c, const double* x, const float2* xhl,
                                                    double* r, CgScalars* cg,
                                                    cudaGraphConditionalHandle h_out) {
    __shared__ double sm[BT / 32];
    double part = 0.0;
    for (int i = blockIdx.x * BT + threadIdx.x; i < c.n; i += gridDim.x * BT) {
        const double dg = c.diag[i];
        double ri = 0.0;
        if (dg != 0.0) {
            const int cnt = c.cnt[i];
            ff acc = {0.f, 0.f};
            const size_t q0 = sell8(i, 0, c.cap);
            const int32_t* cp = c.col + q0;
            const float* hp = c.v32 + q0;
            const float* lp = c.vlo + q0;
            auto term = [&](float ch, float cl, float2 y) {
                ff p = ff_two_prod(ch, y.x);
                p.l = fmaf(ch, y.y, fmaf(cl, y.x, p.l));
                acc = ff_add(acc, p);
            };
            // whole groups of 8 (the last one padded with zeros by the build): columns and
            // both coefficient parts in 16-byte loads, the 8 gathers before their products
            const int ng = (cnt + 7) >> 3;
            for (int g = 0; g < ng; g++) {
                const int4 c0 = *(const int4*)cp, c1 = *(const int4*)(cp + 4);
                const float4 h0 = *(const float4*)hp, h1 = *(const float4*)(hp + 4);
                const float4 l0 = *(const float4*)lp, l1 = *(const float4*)(lp + 4);
                const float2 y0 = xhl[c0.x], y1 = xhl[c0.y], y2 = xhl[c0.z], y3 = xhl[c0.w];
                const float2 y4 = xhl[c1.x], y5 = xhl[c1.y], y6 = xhl[c1.z], y7 = xhl[c1.w];
                term(h0.x, l0.x, y0);
                term(h0.y, l0.y, y1);
                term(h0.z, l0.z, y2);
                term(h0.w, l0.w, y3);
                term(h1.x, l1.x, y4);
                term(h1.y, l1.y, y5);
                term(h1.z, l1.z, y6);
                term(h1.w, l1.w, y7);
                cp += 256;
                hp += 256;
                lp += 256;
            }
            ri = c.bvec[i] - (dg * x[i] - ff_to_double_fast(acc));
        }
        r[i] = ri;
        part = fma(ri, ri, part);
    }
    double tot;
    part = block_sum<BT>(part, sm);
    if (grid_sum<BT>(part, c.partials, &c.counter[0], &tot, sm) && threadIdx.x == 0) {
        cg->rr = tot;
        if (h_out) {
            cg->total += cg->iters;
            cg->outer += 1;
            cg->guard_out += 1;
            const bool more = tot > cg->ostop2 && cg->outer < cg->max_outer &&
                              cg->total < cg->max_total && cg->guard_out < cg->max_outer + 2;
            cudaGraphSetConditional(h_out, more ? 1u : 0u);
        }
    }
}

// start of a solve from x = 0: x = 0, r = b, d = b, rr = rho = b.b, stop2 = tol2 b.b
// h_out (nonzero, the device-driven mixed solve): also the outer target and counters, and
// the refinement loop's conditional (run unless b = 0)
__global__ void __launch_bounds__(kBT) k_start64(SellView c, double* x, double* r, double* d,
                                                 CgScalars* cg, double tol2, float2* xhl,
                                                 cudaGraphConditionalHandle h_out) {
    __shared__ double sm[kWarps];
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < c.n; i += gridDim.x * kBT) {
        const double bi = c.bvec[i];
        x[i] = 0.0;
        if (xhl) xhl[i] = make_float2(0.f, 0.f);
        r[i] = bi;
        d[i] = bi;
        part = fma(bi, bi, part);
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, c.partials, &c.counter[0], &tot, sm) && threadIdx.x == 0) {
        cg->rr = tot;
        cg->stop2 = tol2 * tot;
        cg->rho = tot;
        cg->rho0 = tot;
        cg->done = (tot <= cg->stop2) ? 1 : 0;
        cg->bb = tot;
        if (h_out) {
            cg->ostop2 = tol2 * tot;
            cg->outer = 0;
            cg->total = 0;
            cg->guard_out = 0;
            cudaGraphSetConditional(h_out, tot > cg->ostop2 ? 1u : 0u);
        }
    }
}

// start of a solve from a given guess (cg_x0 = 1), first kernel: bb = b.b and the targets
// tol2 bb of the recurrence and of the refinement; the counters of the device-driven solve
// start one below zero, so that the residual of the guess (the next kernels) is no sweep
__global__ void __launch_bounds__(kBT) k_bnorm64(SellView c, CgScalars* cg, double tol2) {
    __shared__ double sm[kWarps];
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < c.n; i += gridDim.x * kBT)
        part = fma(c.bvec[i], c.bvec[i], part);
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, c.partials, &c.counter[0], &tot, sm) && threadIdx.x == 0) {
        cg->bb = tot;
        cg->stop2 = tol2 * tot;
        cg->ostop2 = tol2 * tot;
        cg->iters = 0;
        cg->outer = -1;
        cg->total = 0;
        cg->guard_out = -1;
    }
}

// second kernel: x = x0 on the rows of the system, 0 elsewhere (and everywhere when b = 0,
// whose solution is 0), with its float-float copy; r = b - A x follows (k_resid64_t or
// k_resid_ff_t).  x0 = sum_k gw[k] h_k over the previous solutions h_0 (latest) to h_3:
// the previous one (weights 1), or its linear (2, -1), quadratic (3, -3, 1) or cubic
// (4, -6, 4, -1) extrapolation in time; a zero weight reads nothing
__global__ void __launch_bounds__(kBT) k_guess(int n, double* x, const double* h0,
                                               const double* h1, const double* h2,
                                               const double* h3, const double* diag,
                                               float2* xhl, const CgScalars* cg) {
    const bool any = cg->bb > 0.0;
    const double w0 = cg->gw[0], w1 = cg->gw[1], w2 = cg->gw[2], w3 = cg->gw[3];
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        double v = 0.0;
        if (any && diag[i] != 0.0) {
            if (w0 != 0.0) v = w0 * h0[i];
            if (w1 != 0.0) v = fma(w1, h1[i], v);
            if (w2 != 0.0) v = fma(w2, h2[i], v);
            if (w3 != 0.0) v = fma(w3, h3[i], v);
        }
        x[i] = v;
        if (xhl) {
            const float h = (float)v;
            xhl[i] = make_float2(h, (float)(v - (double)h));
        }
    }
}

// q = A d, alpha = rho / (d.q)
template <int BT = kBT>
__global__ void __launch_bounds__(BT) k_spmv64_t(SellView c, const double* d, double* q,
                                                  CgScalars* cg) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[BT / 32];
    double part = 0.0;
    for (int i = blockIdx.x * BT + threadIdx.x; i < c.n; i += gridDim.x * BT) {
        const double dg = c.diag[i];
        double qi = 0.0;
        if (dg != 0.0) qi = dg * d[i] - sell_dot64(c, i, d);
        q[i] = qi;
        part = fma(d[i], qi, part);
    }
    double tot;
    part = block_sum<BT>(part, sm);
    if (grid_sum<BT>(part, c.partials, &c.counter[1], &tot, sm) && threadIdx.x == 0) {
        cg->dq = tot;
        cg->alpha = (tot > 0.0) ? cg->rho / tot : 0.0;
    }
}

// FP32 operator: stored FP32 coefficients, or recomputed from the FP32 positions at r*
template <bool MATRIX_FREE, int BT = kBT>
__global__ void __launch_bounds__(BT) k_spmv32_t(SellView c, const float* d, float* q,
                                                 CgScalars* cg, float coef, float re_f) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[BT / 32];
    double part = 0.0;
    for (int i = blockIdx.x * BT + threadIdx.x; i < c.n; i += gridDim.x * BT) {
        const float dg = c.diag32[i];
        float qi = 0.f;
        if (dg != 0.f) {
            const int cnt = c.cnt[i];
            float acc = 0.f;
            if (MATRIX_FREE) {
                const float4 pi = c.pos32s[i];
                for (int k = 0; k < cnt; k++) {
                    const int j = c.col[sell8(i, k, c.cap)];
                    const float4 pj = c.pos32s[j];
                    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    acc = fmaf(coef * fmaf(re_f, rsqrtf(r2), -1.f), d[j], acc);
                }
            } else {
                acc = sell_dot32(c.col + sell8(i, 0, c.cap), c.v32 + sell8(i, 0, c.cap), cnt, d);
            }
            qi = dg * d[i] - acc;
        }
        q[i] = qi;
        part = fma((double)d[i], (double)qi, part);
    }
    double tot;
    part = block_sum<BT>(part, sm);
    if (grid_sum<BT>(part, c.partials, &c.counter[1], &tot, sm) && threadIdx.x == 0) {
        cg->dq = tot;
        cg->alpha = (tot > 0.0) ? cg->rho / tot : 0.0;
    }
}

// ------------------------------------------------------------------ fused inner CG
// The inner CG in two kernels per iteration instead of three, by the recurrences of
// Chronopoulos and Gear (s-step CG, 1989): with w = A r computed from the residual itself,
//   delta_k = (A r_k) . r_k,  beta_k = gamma_k / gamma_{k-1},
//   alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_{k-1})   (alpha_0 = gamma_0/delta_0),
//   p_k = r_k + beta_k p_{k-1},  s_k = w_k + beta_k s_{k-1}  (= A p_k),
//   x += alpha_k p_k,  r_{k+1} = r_k - alpha_k s_k,  gamma_{k+1} = r_{k+1} . r_{k+1}.
// The iterates are those of the textbook CG in exact arithmetic; the vector bytes per
// iteration are the same, one launch and one pass fewer.  p lives in d32, w in q32.
// K1: w = A r and delta; its last block forms alpha (and ends a solve that broke down).
template <bool MATRIX_FREE, int BT = kBT>
__global__ void __launch_bounds__(BT) k_spmv32_cg(SellView c, const float* r, float* w,
                                                  CgScalars* cg, float coef, float re_f) {
    if (*(volatile int*)&cg->done) return;
    __shared__ double sm[BT / 32];
    double part = 0.0;
    for (int i = blockIdx.x * BT + threadIdx.x; i < c.n; i += gridDim.x * BT) {
        const float dg = c.diag32[i];
        float wi = 0.f;
        if (dg != 0.f) {
            const int cnt = c.cnt[i];
            float acc = 0.f;
            if (MATRIX_FREE) {
                const float4 pi = c.pos32s[i];
                for (int k = 0; k < cnt; k++) {
                    const int j = c.col[sell8(i, k, c.cap)];
                    const float4 pj = c.pos32s[j];
                    const float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
                    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                    acc = fmaf(coef * fmaf(re_f, rsqrtf(r2), -1.f), r[j], acc);
                }
            } else {
                acc = sell_dot32(c.col + sell8(i, 0, c.cap), c.v32 + sell8(i, 0, c.cap), cnt, r);
            }
            wi = dg * r[i] - acc;
        }
        w[i] = wi;
        part = fma((double)r[i], (double)wi, part);
    }
    double tot;
    part = block_sum<BT>(part, sm);
    if (grid_sum<BT>(part, c.partials, &c.counter[1], &tot, sm) && threadIdx.x == 0) {
        const bool first = cg->iters == 0;
        const double den = first ? tot : tot - cg->beta * cg->rho / cg->alpha;
        cg->dq = den;
        cg->alpha = (den > 0.0) ? cg->rho / den : 0.0;
        if (!(den > 0.0)) cg->done = 1;
    }
}

// K2: p, s, x and r updated in one pass, gamma of the new residual; its last block forms
// beta and the stop decision.  h_in (nonzero): the inner loop's conditional, set by the last
// block (run again unless done; never more than max_total + 2 times in one inner solve).
__global__ void __launch_bounds__(kBT) k_vec32_cg(int n, float* x, float* r, float* p, float* s,
                                                  const float* w, CgScalars* cg, double* partials,
                                                  unsigned int* counter,
                                                  cudaGraphConditionalHandle h_in) {
    if (*(volatile int*)&cg->done) {
        if (h_in && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h_in, 0u);
        return;
    }
    __shared__ double sm[kWarps];
    const bool first = cg->iters == 0;
    const float alpha = (float)cg->alpha, beta = first ? 0.f : (float)cg->beta;
    double part = 0.0;
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        const float ri = r[i], wi = w[i];
        const float pi = first ? ri : fmaf(beta, p[i], ri);
        const float si = first ? wi : fmaf(beta, s[i], wi);
        p[i] = pi;
        s[i] = si;
        x[i] = fmaf(alpha, pi, x[i]);
        const float rn = fmaf(-alpha, si, ri);
        r[i] = rn;
        part += (double)rn * (double)rn;
    }
    double tot;
    part = block_sum<kBT>(part, sm);
    if (grid_sum<kBT>(part, partials, counter, &tot, sm) && threadIdx.x == 0) {
        cg->beta = (cg->rho > 0.0) ? tot / cg->rho : 0.0;
        cg->rho = tot;
        cg->iters += 1;
        if (tot <= cg->stop2 || cg->iters >= cg->max_iters) cg->done = 1;
        if (h_in) {
            const int g = ++cg->guard_in;
            cudaGraphSetConditional(h_in, (!cg->done && g < cg->max_total + 2) ? 1u : 0u);
        }
    }
}

// x64 += |r64| x32   (|r64| = sqrt(rr) of the residual that started the inner solve); the
// float-float copy of x for the next outer residual is refreshed at the same time
// scale_rr < 0 (the device-driven solve): |r64|^2 is read from the scalars (cg->rr still
// holds the residual that started the inner solve)
__global__ void __launch_bounds__(kBT) k_outer_update(int n, double* x, const float* e, double scale_rr,
                                                      float2* xhl, const CgScalars* cg) {
    const double s = sqrt(scale_rr < 0.0 ? cg->rr : scale_rr);
    for (int i = blockIdx.x * kBT + threadIdx.x; i < n; i += gridDim.x * kBT) {
        const double v = fma(s, (double)e[i], x[i]);
        x[i] = v;
        const float h = (float)v;
        xhl[i] = make_float2(h, (float)(v - (double)h));
    }
}

// Ensemble: |r_s|^2 and |b_s|^2 of every scene (one block per scene over its contiguous
// slot range; deterministic order)
__global__ void __launch_bounds__(kBT) k_scene_sums(const double* r, const double* b,
                                                    const int32_t* cell_start, uint32_t shift,
                                                    double* out) {
    __shared__ double sm[kWarps];
    const int s = blockIdx.x;
    const int lo = cell_start[(size_t)s << shift], hi = cell_start[(size_t)(s + 1) << shift];
    double rr = 0.0, bb = 0.0;
    for (int i = lo + (int)threadIdx.x; i < hi; i += kBT) {
        rr = fma(r[i], r[i], rr);
        bb = fma(b[i], b[i], bb);
    }
    rr = block_sum<kBT>(rr, sm);
    bb = block_sum<kBT>(bb, sm);
    if (threadIdx.x == 0) {
        out[2 * s] = rr;
        out[2 * s + 1] = bb;
    }
}

// Device-driven mixed solve of an ensemble, after each sweep's residual and per-scene sums:
// every scene is checked against cg_tol relative to its own right-hand side once the global
// residual meets the global target; if one is still above, the target is tightened by
// what the worst scene needs (squared, with a margin of 2, within [1e-8, 0.5]); then the
// refinement loop's conditional is set as k_resid_ff_t sets it for a single scene.
__global__ void k_scene_decide(CgScalars* cg, const double* sums, int n_scenes, double tol,
                               cudaGraphConditionalHandle h_out) {
    __shared__ double s_worst[kBT];
    double w = 0.0;
    for (int s = threadIdx.x; s < n_scenes; s += kBT) {
        const double rr = sums[2 * s], bb = sums[2 * s + 1];
        const double rel = bb > 0.0 ? sqrt(rr / bb) : (rr > 0.0 ? HUGE_VAL : 0.0);
        w = fmax(w, rel);
    }
    s_worst[threadIdx.x] = w;
    __syncthreads();
    for (int o = kBT / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_worst[threadIdx.x] = fmax(s_worst[threadIdx.x], s_worst[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    const double worst = s_worst[0];
    cg->total += cg->iters;
    cg->outer += 1;
    cg->guard_out += 1;
    bool more;
    if (cg->rr > cg->ostop2) {
        more = true;
    } else if (worst <= tol) {
        more = false;
    } else {
        const double f = 0.25 * (tol / worst) * (tol / worst);
        cg->ostop2 *= fmin(0.5, fmax(f, 1e-8));
        more = true;
    }
    more = more && cg->outer < cg->max_outer && cg->total < cg->max_total &&
           cg->guard_out < cg->max_outer + 2;
    cg->done = more ? 0 : 1;   // 1: the solve ended (converged or capped)
    cudaGraphSetConditional(h_out, more ? 1u : 0u);
}

// a tighter recurrence target for the FP64 CG (and whether the current residual meets it)
__global__ void k_set_stop(CgScalars* cg, double stop2) {
    cg->stop2 = stop2;
    cg->done = (cg->rho <= stop2) ? 1 : 0;
}

__global__ void k_clear_x(int n, double* x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = 0.0;
}
}  // namespace

// One thread per row, one block per 256 rows (up to the 4096 partial sums of the grid
// reductions; beyond that the row kernels stride): the block scheduler then balances the
// uneven rows (dummy and surface rows are empty) across the SMs.
static int row_grid(const Ctx* c) { return (int)std::min<int64_t>((c->n + kBT - 1) / kBT, 4096); }

static SellView sell_view(Ctx* c, const double* b) {
    SellView v;
    v.n = (int)c->n;
    v.cap = c->cap;
    v.col = c->nb_lap_col;
    v.cnt = c->nb_lap_cnt;
    v.v64 = c->nb_lap_v64;
    v.v32 = c->nb_lap_v32;
    v.vlo = c->nb_lap_vlo;
    v.diag = c->diag;
    v.diag32 = c->diag32;
    v.bvec = b;
    v.pos32s = c->pos32_star;
    v.partials = c->partials;
    v.counter = c->st->counter;
    return v;
}

// Poll the device scalars (one small copy + stream sync).
static int read_scalars(Ctx* c) {
    MPS_CUDA(c, cudaMemcpyAsync(c->cg_host, c->cg, sizeof(CgScalars), cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    return MPS_OK;
}

// Weights of the initial guess over the previous solutions: the highest order the valid
// history allows, up to cg_x0 (1 previous solution, 2 linear, 3 quadratic, 4 cubic
// extrapolation: the polynomial through the last m solutions at equal time steps, taken one
// step further, has the weights (-1)^k C(m, k + 1))
static void guess_weights(const Ctx* c, double* w) {
    static const double kW[5][4] = {{0.0, 0.0, 0.0, 0.0}, {1.0, 0.0, 0.0, 0.0},
                                     {2.0, -1.0, 0.0, 0.0}, {3.0, -3.0, 1.0, 0.0},
                                     {4.0, -6.0, 4.0, -1.0}};
    const int m = std::min(c->guess_n, c->guess_m);
    for (int k = 0; k < 4; k++) w[k] = kW[m][k];
}

static int set_cg_limits(Ctx* c, int max_iters) {
    CgScalars init{};
    init.max_iters = max_iters;
    guess_weights(c, init.gw);
    MPS_CUDA(c, cudaMemcpyAsync(c->cg, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream));
    return MPS_OK;
}

// The FP32 SpMV runs 512-thread blocks: a block's rows are 512 consecutive slots
// (neighbouring particles) that share most of their neighbours, so the gathers of x[col]
// find them in the SM's L1 (256-thread blocks: 5% slower, 128: 25%, 1024: 40%, measured
// on the 3D dam break).  The float-float residual and the FP64 SpMV, with more registers
// and bytes per entry, are faster at 256 (512: 18% and 9% slower).
static int spmv_grid(const Ctx* c, int bt) {
    return (int)std::min<int64_t>((c->n + bt - 1) / bt, 4096);
}

// FP32 SpMV of the inner CG, in the block size the autotuner chose (512: the rows of a block
// are neighbouring particles whose neighbours overlap in L1; 256 on smaller systems)
template <bool MF, int BT>
static void spmv32_bt(Ctx* c, cudaStream_t s, const SellView& sv, bool fused) {
    const float coef = (float)c->coef_ppe, re_f = (float)c->r_lap.re;
    if (fused)
        k_spmv32_cg<MF, BT><<<spmv_grid(c, BT), BT, 0, s>>>(sv, c->cg_r32, c->cg_q32, c->cg, coef, re_f);
    else
        k_spmv32_t<MF, BT><<<spmv_grid(c, BT), BT, 0, s>>>(sv, c->cg_d32, c->cg_q32, c->cg, coef, re_f);
}

static void launch_spmv32(Ctx* c, cudaStream_t s, const SellView& sv, bool fused = false) {
    const bool mf = c->prm.ppe_operator == 1;
    if (c->spmv_block == 256)
        mf ? spmv32_bt<true, 256>(c, s, sv, fused) : spmv32_bt<false, 256>(c, s, sv, fused);
    else
        mf ? spmv32_bt<true, 512>(c, s, sv, fused) : spmv32_bt<false, 512>(c, s, sv, fused);
}

// Launch up to `chunk` iterations of FP64 CG (extra launches exit at once once done).
static void cg64_chunk(Ctx* c, int chunk, double* x, const double* b) {
    const int n = (int)c->n;
    const int gv = vec_grid(c), gs = row_grid(c);
    c->launches += 3 * chunk;
    for (int k = 0; k < chunk; k++) {
        k_spmv64_t<kBT><<<row_grid(c), kBT, 0, c->stream>>>(sell_view(c, b), c->cg_d, c->cg_q, c->cg);
        k_xr64<<<gv, kBT, 0, c->stream>>>(n, x, c->cg_r, c->cg_d, c->cg_q, c->cg, c->partials,
                                          &c->st->counter[2]);
        k_d64<<<gv, kBT, 0, c->stream>>>(n, c->cg_r, c->cg_d, c->cg);
    }
}

static void cg32_chunk(Ctx* c, int chunk, const double* b) {
    const int n = (int)c->n;
    const int gv = vec_grid(c), gs = row_grid(c);
    c->launches += 3 * chunk;
    for (int k = 0; k < chunk; k++) {
        launch_spmv32(c, c->stream, sell_view(c, b));
        k_xr32<<<gv, kBT, 0, c->stream>>>(n, c->cg_x32, c->cg_r32, c->cg_d32, c->cg_q32, c->cg,
                                          c->partials, &c->st->counter[2]);
        k_d32<<<gv, kBT, 0, c->stream>>>(n, c->cg_r32, c->cg_d32, c->cg, 0);
    }
}

// Ensemble: every scene's relative residual from the FP64 residual in cg_r; true when all
// are within cg_tol.  The worst is returned in *worst.
static int scenes_converged(Ctx* c, const double* b, double tol, bool* ok, double* worst) {
    const int S = c->n_scenes;
    k_scene_sums<<<S, kBT, 0, c->stream>>>(c->cg_r, b, c->cell_start, c->scene_shift,
                                           c->scene_sums);
    c->launches += 1;
    std::vector<double> h(2 * (size_t)S);
    MPS_CUDA(c, cudaMemcpyAsync(h.data(), c->scene_sums, sizeof(double) * h.size(),
                                cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    double w = 0.0;
    for (int sc = 0; sc < S; sc++) {
        const double rr = h[2 * sc], bb = h[2 * sc + 1];
        const double rel = bb > 0.0 ? std::sqrt(rr / bb) : (rr > 0.0 ? HUGE_VAL : 0.0);
        c->scene_resid[(size_t)sc] = rel;
        w = std::max(w, rel);
    }
    *ok = w <= tol;
    *worst = w;
    return MPS_OK;
}

// Factor for the global squared-residual target when the worst scene is at `worst` > tol:
// the square of the reduction it still needs, with a margin of 2
static double tighten(double tol, double worst) {
    const double f = 0.25 * (tol / worst) * (tol / worst);
    return std::min(0.5, std::max(f, 1e-8));
}

// ---------------------------------------------------------------- device-driven mixed solve
// The mixed solve of one scene as one CUDA graph:
//   start (x = 0, r = b, outer target)  ->  WHILE (sweeps) {
//       inner init (r32 = r/|r|, tolerance)  ->  WHILE (inner) { A d, x/r update, d update }
//       ->  x += |r| e  ->  r = b - A x (float-float) }
// Both conditions are set by the kernels (one thread each, every iteration), so the solve
// is one launch and one read of the scalars instead of a host poll per chunk of iterations
// and per sweep; the kernels and their arithmetic are those of the host-driven loop, so
// the results are identical.
static cudaGraphNode_t only_node(cudaGraph_t g) {
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> v(nn);
    if (nn) cudaGraphGetNodes(g, v.data(), &nn);
    return nn == 1 ? v[0] : nullptr;
}

static int add_while(Ctx* c, cudaGraph_t g, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                     cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    MPS_CUDA(c, cudaGraphAddNode(node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &cp));
    *body = cp.conditional.phGraph_out[0];
    return MPS_OK;
}

// The mixed solve's nodes appended to graph G after node dep (null: at its root): the start
// sequence, then the WHILE of the refinement sweeps with the WHILE of the inner CG inside.
// *last receives the outer WHILE node.  The scalars (c->cg) must hold their start values
// (mixed_init_scalars) when the nodes run.
int add_mixed_solve(Ctx* c, cudaGraph_t G, cudaGraphNode_t dep, double* x, bool guess,
                    cudaGraphNode_t* last) {
    const int n = (int)c->n;
    const int gs = row_grid(c), gv = vec_grid(c);
    const double tol2 = c->prm.cg_tol * c->prm.cg_tol;
    const SellView sv = sell_view(c, c->bvec);
    cudaStream_t s = c->stream;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaGraph_t B = nullptr, Bi = nullptr, tmp = nullptr;
    cudaGraphConditionalHandle h_out = 0, h_in = 0;
    cudaGraphNode_t n_start, n_outer, n_init, n_inner;
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_out, G, 0, cudaGraphCondAssignDefault));
    const bool multi = c->n_scenes > 1;
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                              mode));
    if (guess) {
        // from the previous solution: b.b, x = x0, r = b - A x and the refinement loop's
        // conditional as after a sweep (per scene in an ensemble)
        k_bnorm64<<<gs, kBT, 0, s>>>(sv, c->cg, tol2);
        k_guess<<<gv, kBT, 0, s>>>(n, x, c->ph[0], c->ph[1], c->ph[2], c->ph[3], c->diag,
                                   c->cg_xhl, c->cg);
        k_resid_ff_t<kBT><<<row_grid(c), kBT, 0, s>>>(sv, x, c->cg_xhl, c->cg_r, c->cg,
                                                      multi ? 0 : h_out);
        if (multi) {
            k_scene_sums<<<c->n_scenes, kBT, 0, s>>>(c->cg_r, c->bvec, c->cell_start,
                                                      c->scene_shift, c->scene_sums);
            k_scene_decide<<<1, kBT, 0, s>>>(c->cg, c->scene_sums, c->n_scenes, c->prm.cg_tol,
                                             h_out);
        }
    } else {
        k_start64<<<gs, kBT, 0, s>>>(sv, x, c->cg_r, c->cg_d, c->cg, tol2, c->cg_xhl, h_out);
    }
    {
        // the last node of the start sequence
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        MPS_CUDA(c, cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
        n_start = (nd == 1) ? deps[0] : nullptr;
    }
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    if (!n_start) return MPS_EDEVICE;
    int rc;
    if ((rc = add_while(c, G, n_start, h_out, &n_outer, &B))) return rc;
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_in, B, 0, cudaGraphCondAssignDefault));
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, B, nullptr, nullptr, 0, mode));
    k_inner_init<<<gv, kBT, 0, s>>>(n, c->cg_r, c->cg_r32, c->cg_d32, c->cg_x32, c->cg, -1.0, 0,
                                    c->partials, &c->st->counter[3], h_in);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    if (!(n_init = only_node(B))) return MPS_EDEVICE;
    if ((rc = add_while(c, B, n_init, h_in, &n_inner, &Bi))) return rc;
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, Bi, nullptr, nullptr, 0, mode));
    // cg_unroll iterations per pass of the loop: once the solve is done the later kernels
    // of the pass return at once (the conditional is set by the last of them)
    for (int u = 0; u < c->cg_unroll; u++) {
        if (c->cg_fused) {
            launch_spmv32(c, s, sv, true);
            k_vec32_cg<<<gv, kBT, 0, s>>>(n, c->cg_x32, c->cg_r32, c->cg_d32, c->cg_s32, c->cg_q32,
                                          c->cg, c->partials, &c->st->counter[2], h_in);
        } else {
            launch_spmv32(c, s, sv);
            k_xr32<<<gv, kBT, 0, s>>>(n, c->cg_x32, c->cg_r32, c->cg_d32, c->cg_q32, c->cg,
                                      c->partials, &c->st->counter[2]);
            k_d32<<<gv, kBT, 0, s>>>(n, c->cg_r32, c->cg_d32, c->cg, h_in);
        }
    }
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, B, &n_inner, nullptr, 1, mode));
    k_outer_update<<<gv, kBT, 0, s>>>(n, x, c->cg_x32, -1.0, c->cg_xhl, c->cg);
    k_resid_ff_t<kBT><<<row_grid(c), kBT, 0, s>>>(sv, x, c->cg_xhl, c->cg_r, c->cg, multi ? 0 : h_out);
    if (multi) {   // every scene to its own tolerance, decided on the device
        k_scene_sums<<<c->n_scenes, kBT, 0, s>>>(c->cg_r, c->bvec, c->cell_start, c->scene_shift,
                                                  c->scene_sums);
        k_scene_decide<<<1, kBT, 0, s>>>(c->cg, c->scene_sums, c->n_scenes, c->prm.cg_tol, h_out);
    }
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    *last = n_outer;
    return MPS_OK;
}

// Start values of the scalars of a device-driven mixed solve: caps, inner tolerance and the
// weights of the initial guess.
void mixed_init_scalars(Ctx* c, CgScalars* init) {
    const int max_total = c->prm.cg_max_iter > 0 ? c->prm.cg_max_iter
                                                 : (int)std::min<int64_t>(10 * c->n, 1 << 30);
    *init = CgScalars{};
    init->max_iters = max_total;
    init->max_total = max_total;
    init->max_outer = c->prm.max_outer > 0 ? c->prm.max_outer : 30;
    init->inner_tol = c->prm.inner_tol;
    guess_weights(c, init->gw);
}

// Kernels one mixed solve ran (counted like the host loop's launches)
int64_t mixed_solve_launches(Ctx* c, bool guess, const CgScalars& h) {
    const bool multi = c->n_scenes > 1;
    // the passes of the inner loop launch cg_unroll iterations each (those after convergence
    // return at once); counted as if the iterations of a solve filled whole passes
    const int64_t u = c->cg_unroll;
    const int64_t inner = (h.total + u - 1) / u * u;
    return (guess ? (multi ? 5 : 3) : 1) + (multi ? 5 : 3) * (int64_t)h.outer +
           (c->cg_fused ? 2 : 3) * inner;
}

namespace {
static int build_mixed_graph(Ctx* c, double* x, PpeGraph* pg) {
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaGraph_t G = nullptr;
    MPS_CUDA(c, cudaGraphCreate(&G, 0));
    pg->graph = G;
    cudaGraphNode_t last = nullptr;
    int rc = add_mixed_solve(c, G, nullptr, x, pg->guess, &last);
    if (rc) {
        abort_capture(c);
        return rc;
    }
    MPS_CUDA(c, cudaGraphInstantiate(&pg->exec, G, 0));
    pg->x = x;
    return MPS_OK;
}
}  // namespace

void ppe_graphs_destroy(Ctx* c) {
    for (PpeGraph& pg : c->ppe_graph) {
        if (pg.exec) cudaGraphExecDestroy(pg.exec);
        if (pg.graph) cudaGraphDestroy(pg.graph);
        pg = PpeGraph{};
    }
}

static int mixed_graph_solve(Ctx* c, double* x, mps_report* rep, int max_total) {
    // keyed by the solution buffer and the guess buffers (all alternate with the bucket build)
    const double* x0 = c->ph[0];
    PpeGraph* pg = nullptr;
    for (PpeGraph& g : c->ppe_graph)
        if (g.exec && g.x == x && g.x0 == x0) pg = &g;
    if (!pg) {
        for (PpeGraph& g : c->ppe_graph)
            if (!g.exec) { pg = &g; break; }
        if (!pg) return MPS_EDEVICE;   // a third buffer pair: not expected
        pg->x0 = x0;
        pg->guess = x0 != nullptr;
        int rc = build_mixed_graph(c, x, pg);
        if (rc) {
            *pg = PpeGraph{};   // the graph of the failed capture is left alone
            c->graphs_off = true;
            return rc;
        }
    }
    CgScalars init;
    mixed_init_scalars(c, &init);
    init.max_iters = init.max_total = max_total;
    MPS_CUDA(c, cudaMemcpyAsync(c->cg, &init, sizeof(CgScalars), cudaMemcpyHostToDevice, c->stream));
    MPS_CUDA(c, cudaGraphLaunch(pg->exec, c->stream));
    int rc;
    if ((rc = read_scalars(c))) return rc;
    const CgScalars h = *c->cg_host;
    const bool multi = c->n_scenes > 1;
    // kernels the graph ran: start, per sweep init + update + residual (+ the per-scene sums
    // and decision of an ensemble), per inner iteration 3
    c->launches += mixed_solve_launches(c, pg->guess, h);
    rep->cg_iters = h.total;
    rep->cg_outer = h.outer;
    c->last_cg_iters = std::max(4, h.total / std::max(h.outer, 1));
    if (!multi) {
        const double rel = h.bb > 0.0 ? sqrt(h.rr / h.bb) : 0.0;
        rep->cg_resid = rel;
        c->scene_resid[0] = rel;
        if (!(h.rr <= h.ostop2)) return MPS_ECG_NOCONV;
        return MPS_OK;
    }
    // ensemble: every scene's residual from the last sweep's per-scene sums
    const int S = c->n_scenes;
    std::vector<double> hs(2 * (size_t)S);
    MPS_CUDA(c, cudaMemcpyAsync(hs.data(), c->scene_sums, sizeof(double) * hs.size(),
                                cudaMemcpyDeviceToHost, c->stream));
    MPS_CUDA(c, cudaStreamSynchronize(c->stream));
    double worst = 0.0;
    for (int sc = 0; sc < S; sc++) {
        const double rr = hs[2 * sc], bb = hs[2 * sc + 1];
        const double rel = bb > 0.0 ? std::sqrt(rr / bb) : (rr > 0.0 ? HUGE_VAL : 0.0);
        c->scene_resid[(size_t)sc] = (h.outer > 0 || pg->guess) ? rel : 0.0;
        worst = std::max(worst, c->scene_resid[(size_t)sc]);
    }
    rep->cg_resid = worst;
    if (!(worst <= c->prm.cg_tol)) return MPS_ECG_NOCONV;
    return MPS_OK;
}

// ---------------------------------------------------------------- kernel timing
// Algorithmic bytes of one launch of the PPE kernels on the current system, summed on the
// device (integers: exact): per row of the system (diag != 0) the stored coefficients and
// the row's own vector entries; per other row the diagonal read and the output write.
__global__ void k_ppe_bytes(int n, const int32_t* cnt, const double* diag, int which,
                            unsigned long long* out) {
    unsigned long long b = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const bool row = diag[i] != 0.0;
        const unsigned long long k = row ? (unsigned long long)cnt[i] : 0ull;
        if (which == 0) b += row ? 8ull * k + 12ull : 8ull;        // col + v32; diag32, d_i, q_i
        else if (which == 1) b += row ? 12ull * k + 32ull : 16ull; // col + v32 + vlo; diag, x_i, b_i, r_i
        else b += row ? 12ull * k + 24ull : 16ull;                 // col + v64; diag, d_i, q_i
    }
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(out, b);
}

int ppe_time_kernel(Ctx* c, int which, int repeats, double* ms, double* bytes) {
    const mps_params& P = c->prm;
    if (P.pressure_mode != 0 || repeats < 1 || which < 0 || which > 2) return MPS_EINVAL;
    if ((which < 2) != (P.precision == 1)) return MPS_EINVAL;
    const int n = (int)c->n;
    const int gs = row_grid(c);
    const SellView sv = sell_view(c, c->bvec);
    cudaStream_t s = c->stream;
    unsigned long long* d_b = (unsigned long long*)c->partials;   // scratch: one word
    MPS_CUDA(c, cudaMemsetAsync(d_b, 0, sizeof(unsigned long long), s));
    k_ppe_bytes<<<c->sms * 4, 256, 0, s>>>(n, c->nb_lap_cnt, c->diag, which, d_b);
    unsigned long long hb = 0;
    MPS_CUDA(c, cudaMemcpyAsync(&hb, d_b, sizeof hb, cudaMemcpyDeviceToHost, s));
    cudaEvent_t e0, e1;
    MPS_CUDA(c, cudaEventCreate(&e0));
    MPS_CUDA(c, cudaEventCreate(&e1));
    float total = 0.f;
    for (int k = 0; k < repeats; k++) {
        // the kernels skip their work once a solve is done: clear the flag (scratch only;
        // the step's results are not touched)
        MPS_CUDA(c, cudaMemsetAsync(&c->cg->done, 0, sizeof(int), s));
        cudaEventRecord(e0, s);
        if (which == 0) {
            launch_spmv32(c, s, sv);
        } else if (which == 1) {
            k_resid_ff_t<kBT><<<row_grid(c), kBT, 0, s>>>(sv, c->p, c->cg_xhl, c->cg_r, c->cg, 0);
        } else {
            k_spmv64_t<kBT><<<row_grid(c), kBT, 0, s>>>(sv, c->cg_d, c->cg_q, c->cg);
        }
        cudaEventRecord(e1, s);
        MPS_CUDA(c, cudaEventSynchronize(e1));
        float m = 0.f;
        cudaEventElapsedTime(&m, e0, e1);
        total += m;
    }
    c->launches += repeats + 1;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    MPS_CUDA(c, cudaGetLastError());
    *ms = total / repeats;
    *bytes = (double)hb;
    return MPS_OK;
}

// A x = b; primary: the step's own PPE (x = p, b = the source), whose iteration count and
// residual the context keeps for the next solve and for mps_scene_residuals
static int solve(Ctx* c, double* x, const double* b, mps_report* rep, bool primary) {
    const int n = (int)c->n;
    const double tol2 = c->prm.cg_tol * c->prm.cg_tol;
    const int max_total = c->prm.cg_max_iter > 0 ? c->prm.cg_max_iter : (int)std::min<int64_t>(10 * c->n, 1 << 30);
    const int gs = row_grid(c), gv = vec_grid(c);
    int rc;
    if (primary && c->prm.precision == 1 && c->prm.ppe_host_loop == 0 && !c->graphs_off)
        return mixed_graph_solve(c, x, rep, max_total);
    if ((rc = set_cg_limits(c, max_total))) return rc;
    // the step's own solve may start from the previous solution (cg_x0 = 1)
    const bool guess = primary && c->guess_m > 0;
    if (guess) {
        // bb = |b|^2, stop2 = tol^2 bb; x = x0; r = b - A x (and d = r, rho = |r|^2 in FP64)
        const SellView sv = sell_view(c, b);
        k_bnorm64<<<gs, kBT, 0, c->stream>>>(sv, c->cg, tol2);
        k_guess<<<gv, kBT, 0, c->stream>>>(n, x, c->ph[0], c->ph[1], c->ph[2], c->ph[3],
                                           c->diag, c->cg_xhl, c->cg);
        if (c->prm.precision == 0)
            k_resid64_t<<<gs, kBT, 0, c->stream>>>(sv, x, c->cg_r, c->cg_d, c->cg, tol2, 0, 1);
        else
            k_resid_ff_t<kBT><<<gs, kBT, 0, c->stream>>>(sv, x, c->cg_xhl, c->cg_r, c->cg, 0);
        c->launches += 3;
    } else {
        // x = 0, r = b, d = b, rho = |b|^2, stop2 = tol^2 |b|^2
        k_start64<<<gs, kBT, 0, c->stream>>>(sell_view(c, b), x, c->cg_r, c->cg_d, c->cg, tol2, c->cg_xhl, 0);
        c->launches += 1;
    }
    if ((rc = read_scalars(c))) return rc;
    const double bnorm2 = guess ? c->cg_host->bb : c->cg_host->rr;
    double stop2 = c->cg_host->stop2;
    int total_iters = 0, outer = 0;
    double rel = 0.0;
    const bool multi = c->n_scenes > 1;
    bool sc_ok = true;
    double sc_worst = 0.0;
    if (multi) std::fill(c->scene_resid.begin(), c->scene_resid.end(), 0.0);
    if (bnorm2 == 0.0) {
        rep->cg_iters = 0;
        rep->cg_outer = 0;
        rep->cg_resid = 0.0;
        return MPS_OK;
    }
    int chunk = std::max(4, c->last_cg_iters + 1);
    if (c->prm.precision == 0) {
        for (;;) {
            cg64_chunk(c, chunk, x, b);
            if ((rc = read_scalars(c))) return rc;
            if (!c->cg_host->done) { chunk = std::max(4, chunk / 2); continue; }
            total_iters = c->cg_host->iters;
            // true residual; restart from it if the recurrence drifted
            c->launches += 1;
            k_resid64_t<<<gs, kBT, 0, c->stream>>>(sell_view(c, b), x, c->cg_r, c->cg_d, c->cg, tol2, 0, 1);
            if ((rc = read_scalars(c))) return rc;
            rel = sqrt(c->cg_host->rr / bnorm2);
            if (c->cg_host->rr <= stop2) {
                if (!multi) break;
                // ensemble: every scene to its own tolerance, else a tighter global target
                if ((rc = scenes_converged(c, b, c->prm.cg_tol, &sc_ok, &sc_worst))) return rc;
                if (sc_ok) break;
                stop2 *= tighten(c->prm.cg_tol, sc_worst);
                k_set_stop<<<1, 1, 0, c->stream>>>(c->cg, stop2);
                c->launches += 1;
            }
            if (total_iters >= max_total) {
                rep->cg_iters = total_iters;
                rep->cg_outer = outer;
                rep->cg_resid = multi ? sc_worst : rel;
                return MPS_ECG_NOCONV;
            }
            outer++;   // restart with the true residual (done was reset by k_resid64)
            chunk = 4;
        }
    } else {
        // mixed: x = 0, r = b (or x = x0, r = b - A x0) already.  Loop: inner FP32 solve,
        // x += e, true residual.
        const int max_outer = c->prm.max_outer > 0 ? c->prm.max_outer : 30;
        double rr = guess ? c->cg_host->rr : bnorm2;
        for (;;) {
            if (rr <= stop2) {
                if (!multi) break;
                // ensemble: every scene to its own tolerance, else a tighter global target
                if ((rc = scenes_converged(c, b, c->prm.cg_tol, &sc_ok, &sc_worst))) return rc;
                if (sc_ok) break;
                stop2 *= tighten(c->prm.cg_tol, sc_worst);
            }
            if (outer >= max_outer || total_iters >= max_total) {
                rep->cg_iters = total_iters;
                rep->cg_outer = outer;
                rep->cg_resid = multi ? sc_worst : sqrt(rr / bnorm2);
                return MPS_ECG_NOCONV;
            }
            // inner reduction: exactly what the outer target still needs (with a margin of 2)
            // when one FP32 solve can reach it, so that the sweep that can finish does so
            // without overshooting; inner_tol for the sweeps before it
            const double need = 0.5 * std::sqrt(stop2 / rr);
            const double itol_k = (need >= kInnerFloor) ? need : c->prm.inner_tol;
            c->launches += 3;
            k_inner_init<<<gv, kBT, 0, c->stream>>>(n, c->cg_r, c->cg_r32, c->cg_d32, c->cg_x32, c->cg,
                                                    itol_k * itol_k, max_total - total_iters,
                                                    c->partials, &c->st->counter[3], 0);
            for (;;) {
                cg32_chunk(c, chunk, b);
                if ((rc = read_scalars(c))) return rc;
                if (c->cg_host->done) break;
                chunk = std::max(4, chunk / 2);
            }
            total_iters += c->cg_host->iters;
            k_outer_update<<<gv, kBT, 0, c->stream>>>(n, x, c->cg_x32, rr, c->cg_xhl, c->cg);
            k_resid_ff_t<kBT><<<row_grid(c), kBT, 0, c->stream>>>(sell_view(c, b), x, c->cg_xhl, c->cg_r, c->cg, 0);
            if ((rc = read_scalars(c))) return rc;
            rr = c->cg_host->rr;
            outer++;
        }
        rel = sqrt(rr / bnorm2);
    }
    if (primary)
        c->last_cg_iters = (c->prm.precision == 0) ? total_iters : std::max(4, total_iters / std::max(outer, 1));
    rep->cg_iters = total_iters;
    rep->cg_outer = outer;
    rep->cg_resid = multi ? sc_worst : rel;   // ensemble: the worst scene
    if (!multi && primary) c->scene_resid[0] = rel;
    MPS_CUDA(c, cudaGetLastError());
    return MPS_OK;
}

int ppe_solve(Ctx* c, mps_report* rep) { return solve(c, c->p, c->bvec, rep, true); }

int ppe_solve_rhs(Ctx* c, double* x, const double* b, mps_report* rep) {
    return solve(c, x, b, rep, false);
}

}  // namespace mps

// ------------------------------------------------------------------ allocation-free solve
// mps_ppe_cg_noalloc: the FP64 CG above on a caller-owned system, with every scratch
// vector, partial sum and scalar taken from one fixed array in device memory that is part
// of the loaded library (so the call itself never allocates).
namespace mps {
namespace {
constexpr int64_t kNoAllocMaxRows = MPS_NOALLOC_MAX_ROWS;
constexpr size_t kNoAllocHead = 512;                       // CgScalars + reduction tickets
constexpr size_t kNoAllocPartials = 4096;                  // per-block partial sums
constexpr int kNoAllocMaxRestarts = 30;                    // true-residual restarts per call
constexpr size_t kNoAllocBytes = kNoAllocHead + kNoAllocPartials * sizeof(double) +
                                 3 * (size_t)kNoAllocMaxRows * sizeof(double);
static_assert(sizeof(CgScalars) <= 256, "CgScalars must fit the scratch header");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_base[kMaxDevices] = {};

// Device address of the scratch array for the current device (resolved once per device).
int noalloc_base(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MPS_EDEVICE;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return MPS_EDEVICE;
        }
        g_noalloc_base[dev] = p;
    }
    *out = g_noalloc_base[dev];
    return MPS_OK;
}

int noalloc_read(CgScalars* host, const CgScalars* dev, cudaStream_t s) {
    if (cudaMemcpyAsync(host, dev, sizeof(CgScalars), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return MPS_EDEVICE;
    if (cudaStreamSynchronize(s) != cudaSuccess) return MPS_EDEVICE;
    return MPS_OK;
}
}  // namespace
}  // namespace mps

extern "C" int mps_ppe_cg_noalloc(int64_t n, int32_t cap, const int32_t* col, const int32_t* cnt,
                                  const double* val, const double* diag, const double* b, double* x,
                                  double tol, int32_t max_iter, void* stream, int32_t* iters_out,
                                  double* resid_out) {
    using namespace mps;
    if (n <= 0 || n > kNoAllocMaxRows || cap <= 0 || !col || !cnt || !val || !diag || !b || !x ||
        !(tol > 0.0))
        return MPS_EINVAL;
    // a launch error left pending by the caller's earlier work is not this call's: report
    // it without clearing it, before launching anything
    if (cudaPeekAtLastError() != cudaSuccess) return MPS_EDEVICE;
    void* base = nullptr;
    int rc = noalloc_base(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* bp = (unsigned char*)base;
    CgScalars* cg = (CgScalars*)bp;
    unsigned int* counters = (unsigned int*)(bp + 256);
    double* partials = (double*)(bp + kNoAllocHead);
    double* r = partials + kNoAllocPartials;
    double* d = r + kNoAllocMaxRows;
    double* q = d + kNoAllocMaxRows;
    const int ni = (int)n;
    const int max_total = max_iter > 0 ? max_iter : (int)std::min<int64_t>(10 * n, 1 << 30);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MPS_EDEVICE;
    // one partial sum per block: the grids never exceed the partials region
    const int gs = std::min(sms * 8, (int)kNoAllocPartials);
    const int gv = std::min(sms * 4, (int)kNoAllocPartials);
    // the array keeps the previous call's contents: scalars and tickets restart from zero
    CgScalars init{};
    init.max_iters = max_total;
    if (cudaMemsetAsync(bp, 0, kNoAllocHead, s) != cudaSuccess ||
        cudaMemcpyAsync(cg, &init, sizeof init, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return MPS_EDEVICE;
    PpeView v;
    v.n = ni;
    v.cap = cap;
    v.col = col;
    v.cnt = cnt;
    v.v64 = val;
    v.v32 = nullptr;
    v.diag = diag;
    v.bvec = b;
    v.pos32s = nullptr;
    v.partials = partials;
    v.counter = counters;
    const double tol2 = tol * tol;
    CgScalars h{};
    k_clear_x<<<(ni + 255) / 256, 256, 0, s>>>(ni, x);
    k_resid64<<<gs, kBT, 0, s>>>(v, x, r, d, cg, tol2, 1, 1);
    if ((rc = noalloc_read(&h, cg, s))) return rc;
    const double bnorm2 = h.rr, stop2 = h.stop2;
    double rel = 0.0;
    int iters = 0;
    int restarts = 0;
    if (bnorm2 > 0.0) {
        int chunk = 8;
        for (;;) {
            if (cudaGetLastError() != cudaSuccess) return MPS_EDEVICE;
            for (int k = 0; k < chunk; k++) {
                k_spmv64<<<gs, kBT, 0, s>>>(v, d, q, cg);
                k_xr64<<<gv, kBT, 0, s>>>(ni, x, r, d, q, cg, partials, &counters[2]);
                k_d64<<<gv, kBT, 0, s>>>(ni, r, d, cg);
            }
            if ((rc = noalloc_read(&h, cg, s))) return rc;
            if (!h.done) continue;
            iters = h.iters;
            k_resid64<<<gs, kBT, 0, s>>>(v, x, r, d, cg, tol2, 0, 1);
            if ((rc = noalloc_read(&h, cg, s))) return rc;
            rel = sqrt(h.rr / bnorm2);
            if (h.rr <= stop2) break;
            // the recurrence met the target but the true residual did not: restart from it,
            // a bounded number of times (a tolerance below what FP64 can attain ends here)
            if (iters >= max_total || ++restarts > kNoAllocMaxRestarts) {
                rc = MPS_ECG_NOCONV;
                break;
            }
        }
    }
    if (cudaGetLastError() != cudaSuccess) return MPS_EDEVICE;
    if (iters_out) *iters_out = iters;
    if (resid_out) *resid_out = rel;
    return rc;
}
