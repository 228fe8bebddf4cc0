// skinpatch.cu -- candidate lists completed by a direct search for the few particles that
// outran the cell skin within a step.
//
// The candidate lists are gathered at r_b (r^k) within max(re)(1 + s) and serve the sums at
// r* as long as no particle moves more than s max(re)/2: then a pair closer than max(re) at
// r* was closer than max(re)(1 + s) at r_b.  When a few particles move farther (the velocity
// spikes of a dam-break surge hitting a wall), only pairs that have one of those "fast"
// particles as an end can be missing.  For each fast particle i every particle j is tested
// at r* (FP32 squared distance below the candidate bound of the full skin: a superset of the
// pairs closer than max(re)), and j is appended to i's list and i to j's list where absent.
// The lists stay supersets without duplicates, so the sums over them -- which decide every
// pair exactly at r* -- are those of complete lists.  A pair of two fast particles is
// entered by each into its own list only (no other block writes a fast particle's list);
// a slow particle's list receives from each fast block only that block's own index, so no
// entry can be appended twice.  More fast particles than the buffer holds (max(64, n/256))
// remains MPS_ESKIN.
#include "mps_internal.cuh"

namespace mps {

namespace {

constexpr int kBT = 256;

// FLUID particles whose |r* - r_b| exceeds half the full skin (the displacement of k_predict)
__global__ void __launch_bounds__(kBT) k_fast_mark(int n, const int32_t* rows, const uint32_t* nrows,
                                                   const double4* pos_star, const double4* pos,
                                                   const double4* pos_b, double half, int cap,
                                                   int32_t* fast, DevStatus* st) {
    const int t = blockIdx.x * kBT + threadIdx.x;
    if (t >= (int)*nrows) return;
    const int i = rows[t];
    const double4 ps = pos_star[i], pb = pos_b ? pos_b[i] : pos[i];
    const double dx = ps.x - pb.x, dy = ps.y - pb.y, dz = ps.z - pb.z;
    const double d2 = fma(dz, dz, fma(dy, dy, dx * dx));
    if (!(sqrt(d2) > half)) return;
    const unsigned q = atomicAdd(&st->n_fast, 1u);
    if ((int)q < cap) fast[q] = i;
}

__device__ __forceinline__ bool in_list(const int32_t* vcol, int row, int cnt, int cap_v, int j) {
    for (int k = 0; k < cnt; k++)
        if (vcol[sell8(row, k, cap_v)] == j) return true;
    return false;
}

__device__ __forceinline__ bool has_row(int t, int dummies) {
    return t == kFluid || t == kWall || (dummies && t == kDummy);
}

// one block per fast particle: every j within the candidate bound at r*
// cnt0: the gathered counts (a copy taken before any append): membership is decided on the
// gathered part of a list, since appended entries (and stale slots beyond the count) can
// only be other blocks' own indices or garbage
__global__ void __launch_bounds__(kBT) k_fast_patch(int n, const int32_t* fast, const DevStatus* stc,
                                                    const float4* p32s, const int8_t* type,
                                                    int32_t* vcol, int32_t* vcnt,
                                                    const int32_t* cnt0, int cap_v, float hv2,
                                                    int dummies, DevStatus* st) {
    const int nf = min((int)stc->n_fast, (int)gridDim.x);
    if ((int)blockIdx.x >= nf) return;
    const int i = fast[blockIdx.x];
    const float4 qi = p32s[i];
    const int cnt_i = min(cnt0[i], cap_v);
    for (int j = threadIdx.x; j < n; j += kBT) {
        if (j == i) continue;
        const int tj = type[j];
        if (tj == kGhost) continue;
        const float4 qj = p32s[j];
        const float dx = qj.x - qi.x, dy = qj.y - qi.y, dz = qj.z - qi.z;
        if (!(fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < hv2)) continue;
        // i's own list (only this block writes it)
        if (!in_list(vcol, i, cnt_i, cap_v, j)) {
            const int s = atomicAdd(&vcnt[i], 1);
            if (s < cap_v) vcol[sell8(i, s, cap_v)] = j;
            else atomicOr(&st->err, kErrCap);
        }
        // j's list, unless j is fast itself (its own block enters i) or has no list
        if (!has_row(tj, dummies)) continue;
        bool j_fast = false;
        for (int f = 0; f < nf && !j_fast; f++) j_fast = fast[f] == j;
        if (j_fast) continue;
        const int cnt_j = min(cnt0[j], cap_v);
        if (!in_list(vcol, j, cnt_j, cap_v, i)) {
            const int s = atomicAdd(&vcnt[j], 1);
            if (s < cap_v) vcol[sell8(j, s, cap_v)] = i;
            else atomicOr(&st->err, kErrCap);
        }
    }
}

}  // namespace

int skin_patch_cap(const Ctx* c) { return (int)std::max<int64_t>(64, c->n / 256); }

void launch_fast_mark(Ctx* c, double half) {
    const int n = (int)c->n;
    k_fast_mark<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(
        n, c->rows_f, c->scan_f + c->n, c->pos_star, c->pos, c->prm.list_every > 1 ? c->pos_b : nullptr,
        half, skin_patch_cap(c), c->fast_idx, c->st);
    c->launches += 1;
}

int launch_fast_patch(Ctx* c, int n_fast, float hv2) {
    if (n_fast <= 0) return MPS_OK;
    // the gathered counts, in the row-mark buffer of the bucket build (free until the next one)
    int32_t* cnt0 = (int32_t*)c->mark_f;
    MPS_CUDA(c, cudaMemcpyAsync(cnt0, c->vl_cnt, sizeof(int32_t) * (size_t)c->n,
                                cudaMemcpyDeviceToDevice, c->stream));
    k_fast_patch<<<n_fast, kBT, 0, c->stream>>>((int)c->n, c->fast_idx, c->st, c->pos32_star,
                                                c->type, c->vl_col, c->vl_cnt, cnt0, c->cap_v,
                                                hv2, c->vjp ? 1 : 0, c->st);
    c->launches += 1;
    return MPS_OK;
}

}  // namespace mps
