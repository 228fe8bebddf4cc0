// gather.cu -- neighbour gathers over the Morton bucket grid (Sec. 4.1: a particle's
// neighbours are looked up in its own cell and the adjacent cells).
//
// One thread block per occupied cell; each thread owns one particle of that cell.  The
// 3^d surrounding cells' particles are staged in shared memory per cell (FP32 positions
// relative to the grid origin and slots, as separate arrays), and every thread walks the
// same staged candidates, two at a time with packed FP32x2 arithmetic, so the shared-memory
// reads are broadcasts and the rare FP64 loads of a candidate are warp-uniform.
//
// Distance predicate of the exact sets: a candidate is classified from its FP32 squared
// distance against a band [lo, hi) around re^2 that bounds the FP32 rounding error; only
// candidates inside the band are decided in binary64 with the exact
// ((dx*dx)+(dy*dy))+(dz*dz) < re*re of the definition, so neighbour sets are identical to
// an FP64 evaluation.
//
// Ops:
//   VerletOp   (r^k): the step's candidate lists, every j within h = max(re)(1 + s) (FP32
//              with a rounding margin: a superset); the pair sums of the step run over
//              these lists (rows.cu).
//   NbrOp      (debug export of exact neighbour sets at r^k).
#include "mps_internal.cuh"

namespace mps {

namespace {

// One block per occupied cell (taken in turn from a device counter), one thread per
// particle of the cell.  The particles of the 3^d surrounding cells (contiguous slot ranges
// in Morton order) are staged in shared memory as (x, y, z, slot) and every thread walks
// the same staged candidates, four per shared-memory load, so each read is a broadcast.
// Staging keeps only candidates within the candidate bound of the block's own cell box (no
// particle of the cell can pair with the others: about a quarter of the 3^d neighbourhood
// in 3D, mostly in the edge and corner cells).  Each warp filters a contiguous part of the
// candidate range into its own segment of the staging buffer (ballot compaction, no block
// barrier), in candidate order, so the lists come out in a fixed order.  One barrier pair
// per cell, more only when the neighbourhood exceeds a chunk.
template <int BT, int CHUNK, class Op>
__global__ void __launch_bounds__(BT)
    k_gather(Op op, const int32_t* __restrict__ cell_start, const uint32_t* __restrict__ occ,
             const DevStatus* st, GridDesc g) {
    constexpr int NW = BT / 32;
    constexpr int WCAP = CHUNK / NW;     // staged entries per warp segment (a multiple of 4)
    constexpr int WRAW = WCAP - 4;       // raw candidates a warp filters per chunk (room for padding)
    static_assert(WCAP % 4 == 0 && WRAW > 0, "chunk too small for the block");
    // staged candidates, structure of arrays: x, y, z relative to the grid origin, slot
    extern __shared__ __align__(16) float s_buf[];
    float* s_x = s_buf;
    float* s_y = s_buf + CHUNK;
    float* s_z = s_buf + 2 * CHUNK;
    int* s_j = (int*)(s_buf + 3 * CHUNK);
    __shared__ int s_cs[27], s_pref[28];
    __shared__ int s_nc;
    __shared__ int s_cnt[NW];
    __shared__ float s_box[7];           // the cell box (lo xyz, hi xyz) and the bound
    const unsigned n_occ = *(volatile const unsigned*)&st->n_occ;
    // an ensemble's keys carry the scene above the cell's Morton code: neighbour cells are
    // looked up under the same prefix, so no gather crosses scenes
    const uint32_t local_mask = (g.dim * g.bits >= 32) ? 0xFFFFFFFFu : ((1u << (g.dim * g.bits)) - 1u);
    __shared__ unsigned s_ci;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (;;) {
        __syncthreads();   // s_ci of the previous cell has been read by every thread
        if (threadIdx.x == 0) s_ci = atomicAdd(&((DevStatus*)st)->gather_next, 1u);
        __syncthreads();
        const unsigned ci = s_ci;
        if (ci >= n_occ) break;
        const uint32_t code = occ[ci];
        const int c0 = cell_start[code], c1 = cell_start[code + 1];
        __syncthreads();   // previous cell's staged data and ranges no longer in use
        if (threadIdx.x == 0) {
            int cc[3];
            const uint32_t prefix = code & ~local_mask;
            morton_decode(code & local_mask, g.dim, g.bits, cc);
            int m = 0, pref = 0;
            const int zr = (g.dim == 3) ? 1 : 0;
            for (int dz = -zr; dz <= zr; dz++)
                for (int dy = -1; dy <= 1; dy++)
                    for (int dx = -1; dx <= 1; dx++) {
                        int nc[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                        if (nc[0] < 0 || nc[1] < 0 || nc[2] < 0 || nc[0] >= g.ncell[0] ||
                            nc[1] >= g.ncell[1] || nc[2] >= g.ncell[2])
                            continue;
                        uint32_t k2 = prefix | morton_encode(nc, g.dim, g.bits);
                        int s0 = cell_start[k2], s1 = cell_start[k2 + 1];
                        if (s1 > s0) {
                            s_cs[m] = s0;
                            s_pref[m] = pref;
                            pref += s1 - s0;
                            m++;
                        }
                    }
            s_pref[m] = pref;
            s_nc = m;
            // the cell box in the FP32 coordinates relative to the grid origin, widened by
            // several roundings of the largest coordinate (a particle's FP32 position may lie
            // just outside its binary64 cell)
            double ext = 0.0;
            for (int a = 0; a < g.dim; a++) ext = fmax(ext, g.ncell[a] * g.h);
            const float eps = (float)(ext * 4.8e-7) + 1e-30f;
            for (int a = 0; a < 3; a++) {
                const bool used = a < g.dim;
                s_box[a] = used ? (float)(cc[a] * g.h) - eps : -eps;
                s_box[3 + a] = used ? (float)((cc[a] + 1) * g.h) + eps : eps;
            }
            s_box[6] = op.block_bound2(c0) * 1.00001f;
        }
        __syncthreads();
        const int ncand = s_pref[s_nc];
        const float4 blo = make_float4(s_box[0], s_box[1], s_box[2], 0.f);
        const float4 bhi = make_float4(s_box[3], s_box[4], s_box[5], 0.f);
        const float bound2 = s_box[6];
        const bool once = ncand <= NW * WRAW;   // whole neighbourhood staged once for the cell
        // filter raw candidates [base, base + len): warp w takes a contiguous part and
        // appends the candidates near the cell box to its segment (padded with sentinels at
        // infinity to a multiple of four, so that the walk needs no tail)
        auto stage = [&](int base, int len) {
            const int per = (len + NW - 1) / NW;
            const int f0 = base + warp * per, f1 = min(base + len, f0 + per);
            float* sx = s_x + warp * WCAP;
            float* sy = s_y + warp * WCAP;
            float* sz = s_z + warp * WCAP;
            int* sj = s_j + warp * WCAP;
            int cnt = 0, m = 0;
            for (int fb = f0; fb < f1; fb += 32) {
                const int f = fb + lane;
                bool keep = false;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                int slot = -1;
                if (f < f1) {
                    while (f >= s_pref[m + 1]) m++;
                    slot = f + s_cs[m] - s_pref[m];
                    q = op.pos32[slot];
                    const float dx = fmaxf(fmaxf(blo.x - q.x, q.x - bhi.x), 0.f);
                    const float dy = fmaxf(fmaxf(blo.y - q.y, q.y - bhi.y), 0.f);
                    const float dz = fmaxf(fmaxf(blo.z - q.z, q.z - bhi.z), 0.f);
                    keep = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < bound2;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, keep);
                if (keep) {
                    const int k = cnt + __popc(bal & ((1u << lane) - 1u));
                    sx[k] = q.x;
                    sy[k] = q.y;
                    sz[k] = q.z;
                    sj[k] = slot;
                }
                cnt += __popc(bal);
            }
            const int padded = (cnt + 3) & ~3;
            if (lane < padded - cnt) {
                sx[cnt + lane] = __int_as_float(0x7f800000);
                sy[cnt + lane] = 0.f;
                sz[cnt + lane] = 0.f;
                sj[cnt + lane] = -1;
            }
            if (lane == 0) s_cnt[warp] = padded;
        };
        if (once) {
            stage(0, ncand);
            __syncthreads();
        }
        for (int ib = c0; ib < c1; ib += BT) {
            const int i = ib + threadIdx.x;
            const bool act = (i < c1) && op.active(i);
            const int nact = __syncthreads_count(act);
            typename Op::Center ctr;
            op.begin(i, act, ctr);
            for (int base = 0; base < ncand; base += NW * WRAW) {
                const int len = min(NW * WRAW, ncand - base);
                if (!once) {
                    if (base > 0 || ib > c0) __syncthreads();   // buffer reuse
                    stage(base, len);
                    __syncthreads();
                }
                if (threadIdx.x == 0 && nact) {
                    int staged = 0;
                    for (int w2 = 0; w2 < NW; w2++) staged += s_cnt[w2];
                    atomicAdd(&((DevStatus*)st)->cand_tests,
                              (unsigned long long)nact * (unsigned long long)staged);
                }
                if (act) {
                    for (int w2 = 0; w2 < NW; w2++) {
                        const int mcnt = s_cnt[w2];
                        const float* sx = s_x + w2 * WCAP;
                        const float* sy = s_y + w2 * WCAP;
                        const float* sz = s_z + w2 * WCAP;
                        const int* sj = s_j + w2 * WCAP;
                        for (int k = 0; k < mcnt; k += 4) {
                            const float4 x4 = *(const float4*)&sx[k], y4 = *(const float4*)&sy[k];
                            const float4 z4 = *(const float4*)&sz[k];
                            const int4 j4 = *(const int4*)&sj[k];
                            op.visit2(ctr, i, make_float2(x4.x, x4.y), make_float2(y4.x, y4.y),
                                      make_float2(z4.x, z4.y), make_int2(j4.x, j4.y));
                            op.visit2(ctr, i, make_float2(x4.z, x4.w), make_float2(y4.z, y4.w),
                                      make_float2(z4.z, z4.w), make_int2(j4.z, j4.w));
                        }
                    }
                }
            }
            op.finish(i, act, ctr);
        }
    }
}

__device__ __forceinline__ float dist2_f(const float4& a, const float4& b) {
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ int kind_of(const float4& q) { return __float_as_int(q.w) & 0xff; }

// ------------------------------------------------------------------------------ Verlet
// Candidate list of every FLUID and WALL particle: all j != i with FP32 squared distance
// below the candidate radius h^2 plus its rounding margin (a superset of the exact set
// within h), written as SELL-32 rows.
struct VerletOp {
    const float4* pos32;
    const int8_t* type;
    DevStatus* st;
    float hv2;
    const float* hv2_dev;   // non-null: the bound is read here (a step graph's control block)
    int cap_v;
    int32_t* vcol;
    int32_t* vcnt;
    const uint16_t* sid;        // ensemble: the scene of every slot (null: one scene)
    const SceneParams* scn;
    int dummies;                // also give DUMMY particles a list (the reverse step)

    struct Center {
        float4 p32;
        float hv2;      // the candidate bound of the particle's scene
        int cnt;
        int32_t* row;   // entry k of this row at row[32 k] (SELL-32)
    };
    // DUMMY particles only ever appear as neighbours: they get no candidate list (unless
    // the reverse step asks for one: their positions enter the number densities)
    __device__ bool active(int i) const {
        const int t = type[i];
        return t == kFluid || t == kWall || (dummies && t == kDummy);
    }
    __device__ void begin(int i, bool act, Center& c) const {
        c.cnt = 0;
        c.row = vcol + sell(i, 0, cap_v);
        c.hv2 = hv2_dev ? *hv2_dev : hv2;
        if (act) {
            c.p32 = pos32[i];
            if (sid) c.hv2 = scn[sid[i]].rv.hi;
        }
    }
    // Branch-free append: a predicated store into the row's next slot.  Past the cap every
    // hit rewrites the last slot (the row is then reported as overflowed by finish()).
    __device__ __forceinline__ void push(Center& c, bool hit, int j) const {
        int32_t* dst = c.row + (size_t)min(c.cnt, cap_v - 1) * 32;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u32 [%0], %1;\n\t}"
            :: "l"(dst), "r"(j), "r"((unsigned)hit));
        c.cnt += hit ? 1 : 0;
    }
    // two candidates with packed FP32x2 arithmetic (each lane of the pair rounds like the
    // scalar dx*dx + dy*dy + dz*dz with fused multiply-adds)
    __device__ __forceinline__ void visit2(Center& c, int i, float2 x, float2 y, float2 z, int2 j) const {
        const float2 dx = __fadd2_rn(x, make_float2(-c.p32.x, -c.p32.x));
        const float2 dy = __fadd2_rn(y, make_float2(-c.p32.y, -c.p32.y));
        const float2 dz = __fadd2_rn(z, make_float2(-c.p32.z, -c.p32.z));
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        push(c, r2.x < c.hv2 && j.x != i, j.x);
        push(c, r2.y < c.hv2 && j.y != i, j.y);
    }
    __device__ void finish(int i, bool act, const Center& c) const {
        if (!act) return;
        vcnt[i] = min(c.cnt, cap_v);
        if (c.cnt > cap_v) atomicOr(&st->err, kErrCap);
    }
    // the candidate bound of the cell's particles (all of one scene), for the staging filter
    __device__ float block_bound2(int i) const {
        if (sid) return scn[sid[i]].rv.hi;
        return hv2_dev ? *hv2_dev : hv2;
    }
};

// ------------------------------------------------------------------------------ debug
struct NbrOp {
    const float4* pos32;
    const double4* pos;
    const int8_t* type;
    const int32_t* id;
    Radius r;
    const int64_t* row_off;
    int32_t* out_ids;
    int32_t* out_cnt;
    struct Center {
        double4 p;
        float4 p32;
        int cnt;
    };
    __device__ bool active(int i) const { return type[i] != kGhost; }
    __device__ void begin(int i, bool act, Center& c) const {
        c.cnt = 0;
        if (!act) return;
        c.p = pos[i];
        c.p32 = pos32[i];
    }
    __device__ void visit(Center& c, int i, int j, const float4& q) const {
        if (j == i) return;
        if (!in_radius(dist2_f(c.p32, q), r, pos, i, j, c.p)) return;
        if (row_off) out_ids[row_off[i] + c.cnt] = id[j];
        c.cnt++;
    }
    __device__ void visit2(Center& c, int i, float2 x, float2 y, float2 z, int2 j) const {
        if (j.x >= 0) visit(c, i, j.x, make_float4(x.x, y.x, z.x, 0.f));
        if (j.y >= 0) visit(c, i, j.y, make_float4(x.y, y.y, z.y, 0.f));
    }
    __device__ void finish(int i, bool act, const Center& c) const {
        if (act && !row_off) out_cnt[i] = c.cnt;
    }
    __device__ float block_bound2(int) const { return r.hi; }
};

__global__ void k_copy_star(int n, const double4* pos, const double4* vel, const float4* pos32,
                            const float4* pos32lo, double4* ps, double4* vs, float4* p32s,
                            float4* p32los) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ps[i] = pos[i];
    vs[i] = vel[i];
    p32s[i] = pos32[i];
    p32los[i] = pos32lo[i];
}

template <int BT, class Op>
void launch_gather_bt(Ctx* c, const Op& op, int blocks_per_sm) {
    // staged candidates per chunk: 512, split evenly over the block's warps (528 for three)
    constexpr int kChunk = (BT == 96) ? 528 : 512;
    // blocks take occupied cells from a counter: cells differ a lot in work (full fluid
    // cells against sparse wall or surface cells), so a static split leaves SMs idle
    cudaMemsetAsync(&c->st->gather_next, 0, sizeof(unsigned int), c->stream);
    k_gather<BT, kChunk, Op><<<c->sms * blocks_per_sm, BT, kChunk * 4 * sizeof(float), c->stream>>>(
        op, c->cell_start, c->occ, c->st, c->grid);
}

template <class Op>
void launch_gather(Ctx* c, const Op& op) {
    c->launches += 1;
    int bt = c->prm.gather_block;
    if (bt == 0) bt = (c->dim == 3) ? 128 : 32;   // measured best on the 3D dam break
    switch (bt) {
        case 32: launch_gather_bt<32>(c, op, 24); break;
        case 64: launch_gather_bt<64>(c, op, 20); break;
        case 128: launch_gather_bt<128>(c, op, 12); break;
        default: launch_gather_bt<96>(c, op, 16); break;
    }
}

}  // namespace

void launch_copy_state_star(Ctx* c) {
    int n = (int)c->n;
    k_copy_star<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->pos, c->vel, c->pos32, c->pos32lo,
                                                         c->pos_star, c->vel_star, c->pos32_star,
                                                         c->pos32lo_star);
    c->launches += 1;
}

void launch_verlet(Ctx* c) {
    VerletOp op;
    op.pos32 = c->pos32;
    op.type = c->type;
    op.st = c->st;
    op.hv2 = c->r_v.hi;
    op.hv2_dev = c->capture_ctl ? &c->capture_ctl->hv2_live : nullptr;
    op.cap_v = c->cap_v;
    op.vcol = c->vl_col;
    op.vcnt = c->vl_cnt;
    op.sid = c->sid;
    op.scn = c->scn;
    op.dummies = c->vjp ? 1 : 0;
    launch_gather<VerletOp>(c, op);
}

void launch_debug_neighbors(Ctx* c, const Radius& r, const int64_t* row_off, int32_t* out_ids,
                            int32_t* out_cnt) {
    NbrOp op;
    op.pos32 = c->pos32;
    op.pos = c->pos;
    op.type = c->type;
    op.id = c->id;
    op.r = r;
    op.row_off = row_off;
    op.out_ids = out_ids;
    op.out_cnt = out_cnt;
    launch_gather<NbrOp>(c, op);
}

}  // namespace mps
