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

// One block per occupied cell (taken in turn from a device counter).  The cell's particles
// that get a list ("active": no DUMMY or GHOST slots; the dummy layers behind the walls fill
// many cells) are compacted, up to NA at a time, with their FP32 positions.  The particles of
// the 3^d surrounding cells (contiguous slot ranges in Morton order) are staged in shared
// memory as (x, y, z, slot), each warp filtering a contiguous part of the candidate range
// into its own segment (ballot compaction, candidate order kept); a candidate is kept only
// within the candidate bound of the bounding box of the compacted actives (taken in the same
// FP32 coordinates as the tests, so no candidate that any of them accepts is dropped: about
// a quarter of the 3^d neighbourhood in full cells, more in thin wall layers and at the free
// surface).  Then the lanes are the candidates: each warp takes pairs of actives in turn and
// tests 32 staged candidates at a time against both (packed FP32x2 arithmetic); the hits of
// each, ranked by a ballot, are appended to its list as one run of consecutive entries in
// candidate order -- with the lists in groups of 8 entries per row (sell8) such a run fills
// whole 32-byte sectors, where one entry per store would write a sector each.
template <int NW, int WCAP, class Op>
__global__ void __launch_bounds__(32 * NW)
    k_gather(Op op, const int32_t* __restrict__ cell_start, const uint32_t* __restrict__ occ,
             const DevStatus* st, GridDesc g) {
    constexpr int NA = 128;              // actives per pass
    constexpr int WRAW = WCAP - 32;      // raw candidates a warp filters per chunk (room for padding)
    static_assert(WRAW >= 128 && WCAP % 32 == 0, "staging segment too small");
    extern __shared__ __align__(16) float4 s_stage[];   // NW segments of WCAP entries
    __shared__ float4 s_ctr[NA];         // the actives: FP32 position, slot in w
    __shared__ int s_len[NA];            // their list lengths so far
    __shared__ int s_cs[27], s_pref[28];
    __shared__ int s_seg[NW], s_kept[NW];   // each segment's padded and kept lengths
    __shared__ float s_box[6];
    __shared__ int s_nact, s_next, s_ncand;
    __shared__ unsigned s_ci[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lane_lt = (1u << lane) - 1u;
    const unsigned n_occ = *(volatile const unsigned*)&st->n_occ;
    // an ensemble's keys carry the scene above the cell's Morton code: neighbour cells are
    // looked up under the same prefix, so no gather crosses scenes
    const uint32_t local_mask = (g.dim * g.bits >= 32) ? 0xFFFFFFFFu : ((1u << (g.dim * g.bits)) - 1u);
    if (threadIdx.x == 0) s_ci[0] = atomicAdd(&((DevStatus*)st)->gather_next, 1u);
    unsigned long long tests = 0;   // candidate tests of this block (counted by thread 0)
    for (int par = 0;; par ^= 1) {
        __syncthreads();   // the cell index is in place; every thread is done with the previous cell
        const unsigned ci = s_ci[par];
        if (ci >= n_occ) break;
        const uint32_t code = occ[ci];
        const int c0 = cell_start[code], c1 = cell_start[code + 1];
        if (warp == NW - 1) {
            // the next cell, fetched while this one is worked on
            if (lane == 0) s_ci[par ^ 1] = atomicAdd(&((DevStatus*)st)->gather_next, 1u);
            // the 3^d neighbour cells, one per lane in the order (dz, dy, dx) = (-1..1)^d,
            // their slot ranges loaded at once; a warp scan gives the staging offsets of the
            // non-empty ones (the same order and offsets as a serial walk over the cells)
            int cc[3];
            const uint32_t prefix = code & ~local_mask;
            morton_decode(code & local_mask, g.dim, g.bits, cc);
            const int ncells_max = (g.dim == 3) ? 27 : 9;
            int s0 = 0, cnt = 0;
            if (lane < ncells_max) {
                const int dx = lane % 3 - 1, dy = (lane / 3) % 3 - 1, dz = (g.dim == 3) ? lane / 9 - 1 : 0;
                int nc[3] = {cc[0] + dx, cc[1] + dy, cc[2] + dz};
                const bool inside = nc[0] >= 0 && nc[1] >= 0 && nc[2] >= 0 && nc[0] < g.ncell[0] &&
                                    nc[1] < g.ncell[1] && nc[2] < g.ncell[2];
                if (inside) {
                    const uint32_t k2 = prefix | morton_encode(nc, g.dim, g.bits);
                    s0 = cell_start[k2];
                    cnt = cell_start[k2 + 1] - s0;
                }
            }
            const bool nonempty = cnt > 0;
            const unsigned bal = __ballot_sync(0xffffffffu, nonempty);
            int incl = cnt;   // inclusive scan of the counts
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            if (nonempty) {
                const int m = __popc(bal & lane_lt);
                s_cs[m] = s0;
                s_pref[m] = incl - cnt;
            }
            if (lane == 31) {
                s_pref[__popc(bal)] = incl;
                s_ncand = incl;
            }
        }
        const float bound2 = op.block_bound2(c0) * 1.00001f;   // the cell's particles share a scene
        for (int a0 = c0; a0 < c1;) {
            if (a0 > c0) __syncthreads();   // the previous pass's actives are no longer read
            if (warp == 0) {
                // compact up to NA active slots of [a0, c1), bounding their FP32 positions
                int nact = 0, a = a0;
                float lx = INFINITY, ly = INFINITY, lz = INFINITY;
                float hx = -INFINITY, hy = -INFINITY, hz = -INFINITY;
                while (a < c1 && nact <= NA - 32) {
                    const int i = a + lane;
                    const bool on = i < c1 && op.active(i);
                    const unsigned bal = __ballot_sync(0xffffffffu, on);
                    if (on) {
                        const float4 q = op.pos32[i];
                        const int k = nact + __popc(bal & lane_lt);
                        s_ctr[k] = make_float4(q.x, q.y, q.z, __int_as_float(i));
                        s_len[k] = 0;
                        lx = fminf(lx, q.x); ly = fminf(ly, q.y); lz = fminf(lz, q.z);
                        hx = fmaxf(hx, q.x); hy = fmaxf(hy, q.y); hz = fmaxf(hz, q.z);
                    }
                    nact += __popc(bal);
                    a += 32;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    lx = fminf(lx, __shfl_xor_sync(0xffffffffu, lx, o));
                    ly = fminf(ly, __shfl_xor_sync(0xffffffffu, ly, o));
                    lz = fminf(lz, __shfl_xor_sync(0xffffffffu, lz, o));
                    hx = fmaxf(hx, __shfl_xor_sync(0xffffffffu, hx, o));
                    hy = fmaxf(hy, __shfl_xor_sync(0xffffffffu, hy, o));
                    hz = fmaxf(hz, __shfl_xor_sync(0xffffffffu, hz, o));
                }
                if (lane == 0) {
                    s_nact = nact;
                    s_next = a;
                    s_box[0] = lx; s_box[1] = ly; s_box[2] = lz;
                    s_box[3] = hx; s_box[4] = hy; s_box[5] = hz;
                }
            }
            __syncthreads();   // actives, box and neighbourhood are in place
            const int nact = s_nact, ncand = s_ncand;
            a0 = s_next;
            if (nact == 0) continue;   // block-uniform
            const float lx = s_box[0], ly = s_box[1], lz = s_box[2];
            const float hx = s_box[3], hy = s_box[4], hz = s_box[5];
            for (int base = 0; base < ncand; base += NW * WRAW) {
                if (base > 0) __syncthreads();   // the previous chunk has been walked
                {
                    // warp w filters the raw candidates [f0, f1) into its segment, four per
                    // lane in flight
                    const int len = min(NW * WRAW, ncand - base);
                    const int per = (len + NW - 1) / NW;
                    const int f0 = base + warp * per, f1 = min(base + len, f0 + per);
                    float4* seg = s_stage + warp * WCAP;
                    int cnt = 0, m = 0;
                    for (int gb = f0; gb < f1; gb += 128) {
                        float4 q[4];
                        int slot[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int f = gb + 32 * u + lane;
                            slot[u] = -1;
                            if (f < f1) {
                                while (f >= s_pref[m + 1]) m++;
                                slot[u] = f + s_cs[m] - s_pref[m];
                                q[u] = op.pos32[slot[u]];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            bool keep = false;
                            if (slot[u] >= 0) {
                                const float dx = fmaxf(fmaxf(lx - q[u].x, q[u].x - hx), 0.f);
                                const float dy = fmaxf(fmaxf(ly - q[u].y, q[u].y - hy), 0.f);
                                const float dz = fmaxf(fmaxf(lz - q[u].z, q[u].z - hz), 0.f);
                                keep = fmaf(dz, dz, fmaf(dy, dy, dx * dx)) < bound2;
                            }
                            const unsigned bal = __ballot_sync(0xffffffffu, keep);
                            if (keep)
                                seg[cnt + __popc(bal & lane_lt)] =
                                    make_float4(q[u].x, q[u].y, q[u].z, __int_as_float(slot[u]));
                            cnt += __popc(bal);
                        }
                    }
                    // padded with sentinels at infinity (no hits) to a multiple of 32 lanes
                    const int padded = (cnt + 31) & ~31;
                    if (cnt + lane < padded)
                        seg[cnt + lane] = make_float4(INFINITY, 0.f, 0.f, __int_as_float(-1));
                    if (lane == 0) {
                        s_seg[warp] = padded;
                        s_kept[warp] = cnt;
                    }
                }
                __syncthreads();   // the chunk is staged
                if (threadIdx.x == 0) {
                    int kept = 0;
                    for (int w2 = 0; w2 < NW; w2++) kept += s_kept[w2];
                    tests += (unsigned long long)nact * (unsigned long long)kept;
                }
                // warp w takes the actives p .. p + 3, p = 4 w, 4 w + 4 NW, ...: one staged
                // candidate per lane, tested against two pairs of them
                for (int p = 4 * warp; p < nact; p += 4 * NW) {
                    typename Op::Center cn[4];
                    int ln[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const bool on = p + t < nact;
                        cn[t] = op.center(s_ctr[on ? p + t : p], on);
                        ln[t] = on ? s_len[p + t] : 0;
                    }
                    for (int w2 = 0; w2 < NW; w2++) {
                        const float4* seg = s_stage + w2 * WCAP;
                        const int padded = s_seg[w2];
                        for (int gk = 0; gk < padded; gk += 32) {
                            const float4 qc = seg[gk + lane];
                            const int j = __float_as_int(qc.w);
                            bool hit[4];
                            op.test2(cn[0], cn[1], qc, j, hit[0], hit[1]);
                            op.test2(cn[2], cn[3], qc, j, hit[2], hit[3]);
#pragma unroll
                            for (int t = 0; t < 4; t++) {
                                const unsigned mt = __ballot_sync(0xffffffffu, hit[t]);
                                if (mt) {   // warp-uniform: a center misses most groups
                                    if (hit[t]) op.put(cn[t], ln[t] + __popc(mt & lane_lt), j);
                                    ln[t] += __popc(mt);
                                }
                            }
                        }
                    }
                    if (lane < 4 && p + lane < nact) {
                        // lane t stores center t's length (registers indexed by a constant)
                        int lv = ln[0];
                        if (lane == 1) lv = ln[1];
                        if (lane == 2) lv = ln[2];
                        if (lane == 3) lv = ln[3];
                        s_len[p + lane] = lv;
                    }
                }
            }
            __syncthreads();   // the lengths are final
            for (int k = threadIdx.x; k < nact; k += 32 * NW)
                op.finish(__float_as_int(s_ctr[k].w), s_len[k]);
        }
    }
    if (threadIdx.x == 0 && tests) atomicAdd(&((DevStatus*)st)->cand_tests, tests);
}

__device__ __forceinline__ float dist2_f(const float4& a, const float4& b) {
    float dx = b.x - a.x, dy = b.y - a.y, dz = b.z - a.z;
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ int kind_of(const float4& q) { return __float_as_int(q.w) & 0xff; }

// ------------------------------------------------------------------------------ Verlet
// Candidate list of every FLUID and WALL particle: all j != i with FP32 squared distance
// below the candidate radius h^2 plus its rounding margin (a superset of the exact set
// within h), written as sell8 rows in candidate order.
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
        float px, py, pz;
        float hv2;      // the candidate bound of the particle's scene (negative: no hits)
        int i;
        size_t row;     // sell8 offset of the row's first entry
    };
    // DUMMY particles only ever appear as neighbours: they get no candidate list (unless
    // the reverse step asks for one: their positions enter the number densities)
    __device__ bool active(int i) const {
        const int t = type[i];
        return t == kFluid || t == kWall || (dummies && t == kDummy);
    }
    __device__ Center center(const float4& c, bool act) const {
        Center r;
        r.px = c.x;
        r.py = c.y;
        r.pz = c.z;
        r.i = __float_as_int(c.w);
        r.row = sell8(r.i, 0, cap_v);
        r.hv2 = !act ? -1.f : sid ? scn[sid[r.i]].rv.hi : (hv2_dev ? *hv2_dev : hv2);
        return r;
    }
    // one candidate against two centers with packed FP32x2 arithmetic (each half rounds like
    // the scalar dx*dx + dy*dy + dz*dz with fused multiply-adds, dx = x_j - x_i)
    __device__ __forceinline__ void test2(const Center& a, const Center& b, const float4& q, int j,
                                          bool& ha, bool& hb) const {
        const float2 dx = __fadd2_rn(make_float2(q.x, q.x), make_float2(-a.px, -b.px));
        const float2 dy = __fadd2_rn(make_float2(q.y, q.y), make_float2(-a.py, -b.py));
        const float2 dz = __fadd2_rn(make_float2(q.z, q.z), make_float2(-a.pz, -b.pz));
        const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
        ha = r2.x < a.hv2 && j != a.i;
        hb = r2.y < b.hv2 && j != b.i;
    }
    // entry k of the row (past the cap the row is reported as overflowed by finish())
    __device__ __forceinline__ void put(const Center& c, int k, int j) const {
        if (k < cap_v) vcol[c.row + (size_t)((k & ~7) * 32 + (k & 7))] = j;
    }
    __device__ void finish(int i, int len) const {
        vcnt[i] = min(len, cap_v);
        if (len > cap_v) atomicOr(&st->err, kErrCap);
    }
    // the candidate bound of the cell's particles (all of one scene), for the staging filter
    __device__ float block_bound2(int i) const {
        if (sid) return scn[sid[i]].rv.hi;
        return hv2_dev ? *hv2_dev : hv2;
    }
};

// ------------------------------------------------------------------------------ debug
// exact neighbour sets at r^k (the FP32 band decided in binary64), as global ids in
// candidate order
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
        int i;
        bool act;
    };
    __device__ bool active(int i) const { return type[i] != kGhost; }
    __device__ Center center(const float4& c, bool act) const {
        Center r_;
        r_.i = __float_as_int(c.w);
        r_.act = act;
        r_.p32 = make_float4(c.x, c.y, c.z, 0.f);
        r_.p = pos[r_.i];
        return r_;
    }
    __device__ bool test(const Center& c, const float4& q, int j) const {
        if (!c.act || j < 0 || j == c.i) return false;
        return in_radius(dist2_f(c.p32, q), r, pos, c.i, j, c.p);
    }
    __device__ void test2(const Center& a, const Center& b, const float4& q, int j, bool& ha,
                          bool& hb) const {
        ha = test(a, q, j);
        hb = test(b, q, j);
    }
    __device__ void put(const Center& c, int k, int j) const {
        if (row_off) out_ids[row_off[c.i] + k] = id[j];
    }
    __device__ void finish(int i, int len) const {
        if (!row_off) out_cnt[i] = len;
    }
    __device__ float block_bound2(int) const { return r.hi; }
};

__global__ void k_copy_star(int n, const double4* pos, const double4* vel, const float4* pos32,
                            const float4* pos32lo, double4* ps, double4* vs, float4* p32s,
                            float4* pff) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ps[i] = pos[i];
    vs[i] = vel[i];
    const float4 h = pos32[i];
    p32s[i] = h;
    pff[2 * i] = h;
    pff[2 * i + 1] = pos32lo[i];
}

template <int NW, class Op>
void launch_gather_nw(Ctx* c, const Op& op, int blocks_per_sm) {
    // each warp stages up to 480 candidates per chunk in its 512-entry segment (8 KB)
    constexpr int kWCAP = 512;
    static_assert(NW * kWCAP * sizeof(float4) <= 48 * 1024, "within the default dynamic shared memory");
    // blocks take occupied cells from a counter: cells differ a lot in work (full fluid
    // cells against sparse wall or surface cells), so a static split leaves SMs idle
    // (a step graph's attempts reset the counter in k_attempt_begin)
    if (!c->capture_ctl) cudaMemsetAsync(&c->st->gather_next, 0, sizeof(unsigned int), c->stream);
    k_gather<NW, kWCAP, Op><<<c->sms * blocks_per_sm, 32 * NW, NW * kWCAP * sizeof(float4), c->stream>>>(
        op, c->cell_start, c->occ, c->st, c->grid);
}

// params.gather_block: threads per cell block (1 to 4 warps)
template <class Op>
void launch_gather(Ctx* c, const Op& op) {
    c->launches += 1;
    int bt = c->prm.gather_block;
    if (bt == 0) bt = (c->dim == 3) ? 128 : 64;
    switch (bt) {
        case 32: launch_gather_nw<1>(c, op, 24); break;
        case 64: launch_gather_nw<2>(c, op, 14); break;
        case 96: launch_gather_nw<3>(c, op, 10); break;
        default: launch_gather_nw<4>(c, op, 8); break;
    }
}

}  // namespace

void launch_copy_state_star(Ctx* c) {
    int n = (int)c->n;
    k_copy_star<<<(n + 255) / 256, 256, 0, c->stream>>>(n, c->pos, c->vel, c->pos32, c->pos32lo,
                                                         c->pos_star, c->vel_star, c->pos32_star,
                                                         c->pff_star);
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
