// bucket.cu -- bucket build of the cell-linked list (Sec. 4.1).
//
// Per step, at the current positions r^k:
//   1. cell key of every particle: c = floor((x - box_min)/h) per axis as in binary64
//      (decided in binary32 where its error bound allows, see cell_floor), Morton
//      interleave (x in bit 0); a particle outside the grid becomes a GHOST and sorts last;
//      in an ensemble the key is prefixed by the particle's scene (scene-major order) and
//      the GHOST test uses the scene's own grid;
//   2. the stable sort of (key, slot): in a graph-run build whose slots are still in the
//      previous build's order, the particles whose key changed are ranked among themselves
//      and merged into that order (below: "the build from the previous order"); otherwise
//      an LSD radix sort with 8-bit digits: per-tile digit histogram, a device-wide
//      exclusive scan of the digit-major histogram table, and a stable scatter that ranks
//      equal digits with warp match masks (both give the same order);
//   3. per-cell counts and their exclusive scan give cell_start (a cell's particles are
//      contiguous in Morton order); occupied cells are collected for the gathers;
//   4. every per-particle array is permuted into the new order (slot s <- old slot perm[s]),
//      the step's predicted state starting as a copy of it (r* := r, u* := u).
#include <cstring>

#include "mps_internal.cuh"

namespace mps {

namespace {
constexpr int kBT = 256;
constexpr int kItems = 8;
constexpr int kTile = kBT * kItems;
constexpr int kRadixBits = 8;
constexpr int kDigits = 1 << kRadixBits;

// Movers (the build from the previous order): mvf non-null records, per slot, whether its
// key differs from the one the slot holds from the previous build, and appends up to
// mov_cap of them as (key, slot) in arbitrary order (their count in st->n_mov).
struct MoverOut {
    uint8_t* mvf;
    uint32_t* key;
    int32_t* slot;
    int cap;
    uint32_t* cnt;   // 4 per mover, zeroed here for the merge's counts
};

__global__ void __launch_bounds__(kBT)
    k_cell_keys(double4* pos, double4* vel, int8_t* type, uint32_t* key, int32_t* slot, int n,
                GridDesc g, DevStatus* st, int mutate, uint32_t outside_key, const uint16_t* sid,
                const SceneParams* scn, uint32_t shift, MoverOut mo) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t old_key = mo.mvf ? key[i] : 0u;
    if (mo.cnt)
        for (int k = i; k < 4 * mo.cap; k += n) mo.cnt[k] = 0u;
    double4 p = pos[i];
    int8_t t = type[i];
    if (mutate) {
        double4 u = vel[i];
        bool fin = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(u.x) &&
                   isfinite(u.y) && isfinite(u.z);
        if (!fin && t != kGhost) atomicOr(&st->err, kErrNonfinite);
    }
    uint32_t k = outside_key;
    if (t != kGhost) {
        int c[3] = {0, 0, 0};
        const double xs[3] = {p.x, p.y, p.z};
        bool inside = true;
        for (int a = 0; a < g.dim; a++) {
            double q = cell_floor(__dsub_rn(xs[a], g.bmin[a]), g.h, g.inv_h, g.inv_hf);
            if (!(q >= 0.0 && q < (double)g.ncell[a])) inside = false;
            else c[a] = (int)q;
        }
        uint32_t prefix = 0;
        if (sid) {
            // ensemble: inside the scene's own grid (its origin, side and cell counts decide
            // GHOSTs as for a scene alone), keyed in the shared grid under the scene's prefix
            const int sc = sid[i];
            const SceneParams& sp = scn[sc];
            for (int a = 0; a < g.dim; a++) {
                const double q = floor(__ddiv_rn(__dsub_rn(xs[a], sp.own_bmin[a]), sp.own_h));
                if (!(q >= 0.0 && q < (double)sp.own_ncell[a])) inside = false;
            }
            prefix = (uint32_t)sc << shift;
        }
        if (inside) {
            k = prefix | morton_encode(c, g.dim, g.bits);
        } else if (mutate) {
            type[i] = kGhost;
            vel[i] = make_double4(0.0, 0.0, 0.0, 0.0);
        }
    }
    if (mutate && k == outside_key) atomicAdd(&st->n_ghost, 1u);
    key[i] = k;
    if (slot) slot[i] = i;
    if (mo.mvf) {
        const bool moved = k != old_key;
        mo.mvf[i] = moved ? 1 : 0;
        if (moved) {
            const unsigned q = atomicAdd(&st->n_mov, 1u);
            if (q < (unsigned)mo.cap) {
                mo.key[q] = k;
                mo.slot[q] = i;
            }
        }
    }
}

// ---------------------------------------------------------------- the build from the
// previous order.  The slots are sorted by their previous keys, with that build's cell table
// (cs: the first slot of every key; the GHOST key, the table size, runs to n).  The stable
// sort of the slots by their new keys -- the order the radix sort gives -- places
//   a slot whose key did not change (a stayer) at s - #(movers m: s_m < s) +
//       #(movers m: (k_m, s_m) < (k, s)): the stayers keep their relative order, and their
//       keys are non-decreasing in slot order;
//   a mover at #(stayers with (key, slot) < (k_m, s_m)) + #(movers before it), where the
//       stayers of smaller keys are the slots before cs[k_m] less the movers among them, and
//       the stayers of key k_m (all within [cs[k_m], cs_end[k_m]), where the mover is not)
//       come before it when it lies after that range.
// Counts between movers are all-pairs over tiles of 256 x 256 (the movers are few).
__device__ __forceinline__ int old_end(const int32_t* cs, uint32_t k, uint32_t ghost_key, int n) {
    return k < ghost_key ? cs[k + 1] : n;
}

__global__ void __launch_bounds__(kBT)
    k_mov_count(const uint32_t* mkey, const int32_t* mslot, const DevStatus* st, int cap,
                const int32_t* cs, uint32_t ghost_key, int n, uint32_t* cnt) {
    const int M = (int)min(st->n_mov, (unsigned)cap);
    const int T = (M + kBT - 1) / kBT;
    __shared__ uint32_t s_k[kBT];
    __shared__ int32_t s_s[kBT];
    for (int t = blockIdx.x; t < T * T; t += gridDim.x) {
        const int ti = t / T, tj = t - ti * T;
        const int i = ti * kBT + threadIdx.x;
        const int jn = min(kBT, M - tj * kBT);
        __syncthreads();
        if ((int)threadIdx.x < jn) {
            s_k[threadIdx.x] = mkey[tj * kBT + threadIdx.x];
            s_s[threadIdx.x] = mslot[tj * kBT + threadIdx.x];
        }
        __syncthreads();
        if (i >= M) continue;
        const uint32_t ki = mkey[i];
        const int si = mslot[i];
        const int a = ki <= ghost_key ? cs[ki] : n;
        const int b = old_end(cs, ki, ghost_key, n);
        uint32_t lt_ks = 0, lt_s = 0, lt_a = 0, in_r = 0;
        for (int j = 0; j < jn; j++) {
            const uint32_t kj = s_k[j];
            const int sj = s_s[j];
            lt_ks += (kj < ki || (kj == ki && sj < si)) ? 1u : 0u;
            lt_s += sj < si ? 1u : 0u;
            lt_a += sj < a ? 1u : 0u;
            in_r += (sj >= a && sj < b) ? 1u : 0u;
        }
        atomicAdd(&cnt[4 * i + 0], lt_ks);
        atomicAdd(&cnt[4 * i + 1], lt_s);
        atomicAdd(&cnt[4 * i + 2], lt_a);
        atomicAdd(&cnt[4 * i + 3], in_r);
    }
}

__global__ void __launch_bounds__(kBT)
    k_mov_place(const uint32_t* mkey, const int32_t* mslot, const DevStatus* st, int cap,
                const int32_t* cs, uint32_t ghost_key, int n, const uint32_t* cnt,
                int32_t* by_slot, unsigned long long* by_key, uint32_t* kout, int32_t* vout) {
    const int M = (int)min(st->n_mov, (unsigned)cap);
    for (int i = blockIdx.x * kBT + threadIdx.x; i < M; i += gridDim.x * kBT) {
        const uint32_t ki = mkey[i];
        const int si = mslot[i];
        const int a = cs[ki];
        const int b = old_end(cs, ki, ghost_key, n);
        const uint32_t lt_ks = cnt[4 * i + 0], lt_s = cnt[4 * i + 1];
        const uint32_t lt_a = cnt[4 * i + 2], in_r = cnt[4 * i + 3];
        const int stay_before = (a - (int)lt_a) + (si >= b ? (b - a) - (int)in_r : 0);
        const int dst = stay_before + (int)lt_ks;
        by_slot[lt_s] = si;
        by_key[lt_ks] = ((unsigned long long)ki << 32) | (unsigned)si;
        kout[dst] = ki;
        vout[dst] = si;
    }
}

// first index in v[0, m) not below x
template <class T>
__device__ __forceinline__ int lower_bound(const T* v, int m, T x) {
    int lo = 0, hi = m;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kBT)
    k_stay_place(const uint32_t* kin, const uint8_t* mvf, int n, const DevStatus* st, int cap,
                 const int32_t* by_slot, const unsigned long long* by_key, uint32_t* kout,
                 int32_t* vout) {
    const int s = blockIdx.x * kBT + threadIdx.x;
    if (s >= n || mvf[s]) return;
    const int M = (int)min(st->n_mov, (unsigned)cap);
    const uint32_t k = kin[s];
    int dst = s;
    if (M > 0) {
        dst += lower_bound(by_key, M, ((unsigned long long)k << 32) | (unsigned)s) -
               lower_bound(by_slot, M, (int32_t)s);
    }
    kout[dst] = k;
    vout[dst] = s;
}

// the branch of this build: the radix sort unless the previous order holds (the host's
// word) and every mover was recorded
__global__ void k_bucket_branch(const DevStatus* st, const int32_t* order_ok, int cap,
                                cudaGraphConditionalHandle h_radix, cudaGraphConditionalHandle h_inc) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const bool inc = *order_ok != 0 && st->n_mov <= (unsigned)cap;
    cudaGraphSetConditional(h_radix, inc ? 0u : 1u);
    cudaGraphSetConditional(h_inc, inc ? 1u : 0u);
}

__global__ void __launch_bounds__(kBT)
    k_radix_hist(const uint32_t* keys, int n, int shift, uint32_t* hist) {
    __shared__ uint32_t s_h[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kBT) s_h[d] = 0;
    __syncthreads();
    const int base = blockIdx.x * kTile;
    for (int r = 0; r < kItems; r++) {
        int i = base + r * kBT + threadIdx.x;
        if (i < n) atomicAdd(&s_h[(keys[i] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kBT) hist[(size_t)d * gridDim.x + blockIdx.x] = s_h[d];
}

// Stable scatter: the tile is visited in rounds of kBT consecutive keys; within a round a
// key's rank among equal digits is (equal digits in earlier warps) + (equal digits in
// earlier lanes of its own warp), on top of the running per-digit offset of the tile.
__global__ void __launch_bounds__(kBT)
    k_radix_scatter(const uint32_t* kin, const int32_t* vin, uint32_t* kout, int32_t* vout, int n,
                    int shift, const uint32_t* offsets) {
    __shared__ uint32_t s_off[kDigits];
    __shared__ uint32_t s_wc[kBT / 32][kDigits];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int d = threadIdx.x; d < kDigits; d += kBT) s_off[d] = offsets[(size_t)d * gridDim.x + blockIdx.x];
    const int base = blockIdx.x * kTile;
    for (int r = 0; r < kItems; r++) {
        for (int q = threadIdx.x; q < (kBT / 32) * kDigits; q += kBT) (&s_wc[0][0])[q] = 0;
        __syncthreads();
        int i = base + r * kBT + threadIdx.x;
        bool valid = i < n;
        uint32_t k = valid ? kin[i] : 0u;
        int32_t v = valid ? vin[i] : 0;
        int d = valid ? (int)((k >> shift) & (kDigits - 1)) : kDigits;   // sentinel digit
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank = __popc(peers & lt);
        if (valid && rank == 0) s_wc[w][d] = __popc(peers);
        __syncthreads();
        uint32_t tot = 0;
        for (int dd = threadIdx.x; dd < kDigits; dd += kBT) {
            uint32_t run = 0;
            for (int ww = 0; ww < kBT / 32; ww++) {
                uint32_t cnt = s_wc[ww][dd];
                s_wc[ww][dd] = run;
                run += cnt;
            }
            tot = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = s_off[d] + s_wc[w][d] + (uint32_t)rank;
            kout[dst] = k;
            vout[dst] = v;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kDigits; dd += kBT) s_off[dd] += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kBT)
    k_cell_count(const uint32_t* key, int n, uint32_t ghost_key, uint32_t* count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && key[i] != ghost_key) atomicAdd(&count[key[i]], 1u);
}

// cell_start[c] = the number of sorted keys below c, for c = 0 .. ntable (the GHOST key is
// ntable): a binary search per cell, where the table is not much larger than the particle
// count (the counts and their scan are used otherwise; both give the same table)
__global__ void __launch_bounds__(kBT)
    k_cell_start_search(const uint32_t* key, int n, int64_t ntable, int32_t* cell_start) {
    for (int64_t c = blockIdx.x * (int64_t)kBT + threadIdx.x; c <= ntable;
         c += (int64_t)gridDim.x * kBT) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((int64_t)key[mid] < c) lo = mid + 1;
            else hi = mid;
        }
        cell_start[c] = lo;
    }
}

// first slot of each run of equal keys (sorted) marks an occupied cell
__global__ void __launch_bounds__(kBT)
    k_occupied(const uint32_t* key, int n, uint32_t ghost_key, uint32_t* occ, DevStatus* st) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = key[i];
    if (k == ghost_key) return;
    if (i == 0 || key[i - 1] != k) {
        unsigned int q = atomicAdd(&st->n_occ, 1u);
        occ[q] = k;
    }
}

// the previous PPE solutions (cg_x0 >= 1) follow their particles
struct GuessPerm {
    const double* in[Ctx::kGuessMax];
    double* out[Ctx::kGuessMax];
    int m;
};

// the step's predicted state starts as r* = r, u* = u (the prediction overwrites the FLUID
// rows): written here with the permuted state instead of by a separate copy
struct StarOut {
    double4 *pos, *vel;
    float4 *pos32, *pff;   // pff: (hi, lo) pairs, slot s at 2 s and 2 s + 1
    int32_t* vcnt;         // candidate-list counts, zeroed (the gather writes its particles')
};

__global__ void __launch_bounds__(kBT)
    k_permute(const int32_t* perm, int n, const double4* pos, const double4* vel,
              const int8_t* type, const int32_t* id, const double* p, double4* pos_o,
              double4* vel_o, int8_t* type_o, int32_t* id_o, double* p_o, GuessPerm gp,
              float4* pos32, float4* pos32lo, float4* vel32, GridDesc g, StarOut so,
              uint32_t* blk_f, uint32_t* blk_fw) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    // the block's FLUID and FLUID / WALL slots of the new order, counted for the row lists
    {
        __shared__ uint32_t s_cf[kBT / 32], s_cfw[kBT / 32];
        const int tt = s < n ? (int)type[perm[s]] : -1;
        const unsigned bf = __ballot_sync(0xffffffffu, tt == kFluid);
        const unsigned bfw = __ballot_sync(0xffffffffu, tt == kFluid || tt == kWall);
        if ((threadIdx.x & 31) == 0) {
            s_cf[threadIdx.x >> 5] = __popc(bf);
            s_cfw[threadIdx.x >> 5] = __popc(bfw);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t a = 0, b = 0;
            for (int w = 0; w < kBT / 32; w++) {
                a += s_cf[w];
                b += s_cfw[w];
            }
            blk_f[blockIdx.x] = a;
            blk_fw[blockIdx.x] = b;
        }
    }
    if (s >= n) return;
    int j = perm[s];
    double4 x = pos[j];
    int8_t t = type[j];
    const double4 u = vel[j];
    pos_o[s] = x;
    vel_o[s] = u;
    vel32[s] = make_float4((float)u.x, (float)u.y, (float)u.z, 0.f);
    type_o[s] = t;
    id_o[s] = id[j];
    p_o[s] = p[j];
    for (int k = 0; k < gp.m; k++) gp.out[k][s] = gp.in[k][j];   // the PPE guess history
    float4 h, l;
    split_rel(x.x, g.bmin[0], &h.x, &l.x);
    split_rel(x.y, g.bmin[1], &h.y, &l.y);
    split_rel(x.z, g.bmin[2], &h.z, &l.z);
    h.w = __int_as_float((int)t);
    l.w = 0.f;
    pos32[s] = h;
    pos32lo[s] = l;
    so.pos[s] = x;
    so.vel[s] = u;
    so.pos32[s] = h;
    so.pff[2 * s] = h;
    so.pff[2 * s + 1] = l;
    so.vcnt[s] = 0;
}
// The row lists of the new order (FLUID slots, FLUID / WALL slots, each in slot order) from
// the permutation's per-block counts: an exclusive scan of the counts in one block (their
// totals are the lists' lengths, stored after the n entries of scan_f / scan_fw), then every
// block places its slots at its offset plus their rank in the block (warp ballots).
constexpr int kScanBT = 1024;
__global__ void __launch_bounds__(kScanBT)
    k_rows_scan(int nb, uint32_t* blk_f, uint32_t* blk_fw, uint32_t* total_f,
                uint32_t* total_fw) {
    __shared__ uint32_t s_w[2][kScanBT / 32];
    __shared__ uint32_t s_carry[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_carry[0] = s_carry[1] = 0u;
    __syncthreads();
    for (int base = 0; base < nb; base += kScanBT) {
        const int k = base + (int)threadIdx.x;
        uint32_t v[2] = {k < nb ? blk_f[k] : 0u, k < nb ? blk_fw[k] : 0u};
        uint32_t incl[2] = {v[0], v[1]};
        for (int o = 1; o < 32; o <<= 1) {
            for (int a = 0; a < 2; a++) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl[a], o);
                if (lane >= o) incl[a] += y;
            }
        }
        if (lane == 31) {
            s_w[0][w] = incl[0];
            s_w[1][w] = incl[1];
        }
        __syncthreads();
        if (w == 0) {
            for (int a = 0; a < 2; a++) {
                uint32_t t = s_w[a][lane];
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                s_w[a][lane] = t;   // inclusive over the warps
            }
        }
        __syncthreads();
        for (int a = 0; a < 2; a++) {
            const uint32_t before = s_carry[a] + (w > 0 ? s_w[a][w - 1] : 0u);
            if (k < nb) (a == 0 ? blk_f : blk_fw)[k] = before + incl[a] - v[a];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_carry[0] += s_w[0][kScanBT / 32 - 1];
            s_carry[1] += s_w[1][kScanBT / 32 - 1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *total_f = s_carry[0];
        *total_fw = s_carry[1];
    }
}

__global__ void __launch_bounds__(kBT)
    k_rows_scatter(int n, const int8_t* type, const uint32_t* off_f, const uint32_t* off_fw,
                   int32_t* rows_f, int32_t* rows_fw) {
    __shared__ uint32_t s_cf[kBT / 32], s_cfw[kBT / 32];
    const int s = blockIdx.x * kBT + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int t = s < n ? (int)type[s] : -1;
    const bool f = t == kFluid, fw = t == kFluid || t == kWall;
    const unsigned bf = __ballot_sync(0xffffffffu, f), bfw = __ballot_sync(0xffffffffu, fw);
    if (lane == 0) {
        s_cf[w] = __popc(bf);
        s_cfw[w] = __popc(bfw);
    }
    __syncthreads();
    uint32_t of = off_f[blockIdx.x], ofw = off_fw[blockIdx.x];
    for (int k = 0; k < w; k++) {
        of += s_cf[k];
        ofw += s_cfw[k];
    }
    const unsigned lt = (1u << lane) - 1u;
    if (f) rows_f[of + __popc(bf & lt)] = s;
    if (fw) rows_fw[ofw + __popc(bfw & lt)] = s;
}
}  // namespace

void launch_cell_keys_only(Ctx* c, uint32_t* out_key) {
    int n = (int)c->n;
    // exported keys mark particles outside the grid (and GHOSTs) with 0xFFFFFFFF
    k_cell_keys<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(c->pos, c->vel, c->type, out_key,
                                                             nullptr, n, c->grid, c->st, 0,
                                                             0xFFFFFFFFu, nullptr, nullptr, 0,
                                                             MoverOut{});
    c->launches += 1;
}

namespace {
// ---- the stages of a bucket build (each adds its kernels to c->launches)
void launch_keys(Ctx* c, bool mutate, bool movers) {
    const int n = (int)c->n;
    MoverOut mo{};
    if (movers) mo = MoverOut{c->mvf, c->mov_key, c->mov_slot, c->mov_cap, c->mov_cnt};
    k_cell_keys<<<(n + kBT - 1) / kBT, kBT, 0, c->stream>>>(
        c->pos, c->vel, c->type, c->key, c->perm, n, c->grid, c->st, mutate ? 1 : 0,
        c->grid.ghost_key, c->sid, c->scn, c->scene_shift, mo);
    c->launches += 1;
}

// LSD radix sort of (c->key, c->perm) over sort_bits; afterwards c->key and c->perm name
// the buffers holding the sorted keys and the permutation
void launch_radix(Ctx* c) {
    const int n = (int)c->n;
    cudaStream_t s = c->stream;
    const int nt = (n + kTile - 1) / kTile;
    uint32_t* kin = c->key;
    int32_t* vin = c->perm;
    uint32_t* kout = c->key_alt;
    int32_t* vout = c->perm_alt;
    for (int shift = 0; shift < c->sort_bits; shift += kRadixBits) {
        k_radix_hist<<<nt, kBT, 0, s>>>(kin, n, shift, c->hist);
        c->launches += 2 + scan_exclusive(c->hist, c->hist_scan, (int64_t)kDigits * nt, false,
                                          c->scan_scratch, s);
        k_radix_scatter<<<nt, kBT, 0, s>>>(kin, vin, kout, vout, n, shift, c->hist_scan);
        uint32_t* tk = kin; kin = kout; kout = tk;
        int32_t* tv = vin; vin = vout; vout = tv;
    }
    if (kin != c->key) { c->key_alt = c->key; c->key = kin; }
    if (vin != c->perm) { c->perm_alt = c->perm; c->perm = vin; }
}

// the build from the previous order: the new keys (slot order) in kin, the sorted keys and
// the permutation into kout / vout (kout != kin)
int launch_from_previous(Ctx* c, const uint32_t* kin, uint32_t* kout, int32_t* vout) {
    const int n = (int)c->n;
    cudaStream_t s = c->stream;
    const uint32_t gk = c->grid.ghost_key;
    k_mov_count<<<c->sms * 4, kBT, 0, s>>>(c->mov_key, c->mov_slot, c->st, c->mov_cap,
                                           c->cell_start, gk, n, c->mov_cnt);
    k_mov_place<<<(c->mov_cap + kBT - 1) / kBT, kBT, 0, s>>>(
        c->mov_key, c->mov_slot, c->st, c->mov_cap, c->cell_start, gk, n, c->mov_cnt,
        c->mov_by_slot, c->mov_by_key, kout, vout);
    k_stay_place<<<(n + kBT - 1) / kBT, kBT, 0, s>>>(kin, c->mvf, n, c->st, c->mov_cap,
                                                     c->mov_by_slot, c->mov_by_key, kout, vout);
    c->launches += 3;
    return MPS_OK;
}

// cell table of the sorted keys, the state permuted into the new order (and r* := r), the
// active-row lists, the two-phase properties
int launch_table_rest(Ctx* c) {
    const int n = (int)c->n;
    cudaStream_t s = c->stream;
    const int nb1 = (n + kBT - 1) / kBT;
    if (c->ntable <= 2 * (int64_t)n) {
        const int64_t nbt = (c->ntable + 1 + kBT - 1) / kBT;
        k_cell_start_search<<<(int)std::min<int64_t>(nbt, (int64_t)c->sms * 16), kBT, 0, s>>>(
            c->key, n, c->ntable, c->cell_start);
        c->launches += 3;
    } else {
        MPS_CUDA(c, cudaMemsetAsync(c->cell_count, 0, sizeof(uint32_t) * (size_t)c->ntable, s));
        k_cell_count<<<nb1, kBT, 0, s>>>(c->key, n, c->grid.ghost_key, c->cell_count);
        c->launches += 3 + scan_exclusive(c->cell_count, (uint32_t*)c->cell_start, c->ntable,
                                          true, c->scan_scratch, s);
    }
    k_occupied<<<nb1, kBT, 0, s>>>(c->key, n, c->grid.ghost_key, c->occ, c->st);
    // permute the state into the new order
    GuessPerm gp{};
    gp.m = c->guess_m;
    for (int k = 0; k < c->guess_m; k++) {
        gp.in[k] = c->ph[k];
        gp.out[k] = c->ph_alt[k];
    }
    k_permute<<<nb1, kBT, 0, s>>>(c->perm, n, c->pos, c->vel, c->type, c->id, c->p, c->pos_alt,
                                  c->vel_alt, c->type_alt, c->id_alt, c->p_alt, gp, c->pos32,
                                  c->pos32lo, c->vel32, c->grid,
                                  StarOut{c->pos_star, c->vel_star, c->pos32_star, c->pff_star,
                                          c->vl_cnt},
                                  c->mark_f, c->mark_fw);
    std::swap(c->pos, c->pos_alt);
    std::swap(c->vel, c->vel_alt);
    std::swap(c->type, c->type_alt);
    std::swap(c->id, c->id_alt);
    std::swap(c->p, c->p_alt);
    for (int k = 0; k < c->guess_m; k++) std::swap(c->ph[k], c->ph_alt[k]);
    // FLUID rows and FLUID / WALL rows in slot order, for the per-row kernels (the
    // permutation's per-block counts in mark_f / mark_fw, free until the next build)
    k_rows_scan<<<1, kScanBT, 0, s>>>(nb1, c->mark_f, c->mark_fw, c->scan_f + n, c->scan_fw + n);
    k_rows_scatter<<<nb1, kBT, 0, s>>>(n, c->type, c->mark_f, c->mark_fw, c->rows_f, c->rows_fw);
    c->launches += 2;
    launch_gather_props(c);   // two-phase properties follow their particles
    MPS_CUDA(c, cudaGetLastError());
    return MPS_OK;
}

// launch by launch: always the radix sort
int bucket_launches(Ctx* c, bool mutate) {
    launch_keys(c, mutate, false);
    launch_radix(c);
    int rc = launch_table_rest(c);
    if (!rc) c->order_valid = true;
    c->last_bucket_merged = 0;
    return rc;
}

// The bucket build is ~25 short dependent kernels whose launch gaps cost more than their
// work, so the stepping path replays it as one CUDA graph.  Every build swaps the state with
// its alternate buffers (and the radix sort's keys and permutation with theirs when it
// takes an odd number of passes), so there are two graphs, keyed by the position buffer
// the build starts from; each remembers the buffer assignment its build leaves behind.
struct BucketPtrs {
    uint32_t *key, *key_alt;
    int32_t *perm, *perm_alt;
    double4 *pos, *pos_alt, *vel, *vel_alt;
    int8_t *type, *type_alt;
    int32_t *id, *id_alt;
    double *p, *p_alt;
    double *ph[Ctx::kGuessMax], *ph_alt[Ctx::kGuessMax];
};
BucketPtrs save_ptrs(const Ctx* c) {
    return {c->key, c->key_alt, c->perm, c->perm_alt, c->pos, c->pos_alt, c->vel, c->vel_alt,
            c->type, c->type_alt, c->id, c->id_alt, c->p, c->p_alt,
            {c->ph[0], c->ph[1], c->ph[2], c->ph[3]},
            {c->ph_alt[0], c->ph_alt[1], c->ph_alt[2], c->ph_alt[3]}};
}
void load_ptrs(Ctx* c, const BucketPtrs& b) {
    c->key = b.key; c->key_alt = b.key_alt; c->perm = b.perm; c->perm_alt = b.perm_alt;
    c->pos = b.pos; c->pos_alt = b.pos_alt; c->vel = b.vel; c->vel_alt = b.vel_alt;
    c->type = b.type; c->type_alt = b.type_alt; c->id = b.id; c->id_alt = b.id_alt;
    c->p = b.p; c->p_alt = b.p_alt;
    for (int k = 0; k < Ctx::kGuessMax; k++) {
        c->ph[k] = b.ph[k];
        c->ph_alt[k] = b.ph_alt[k];
    }
}
}  // namespace

void state_ptrs_save(const Ctx* c, void* rec) {
    static_assert(sizeof(BucketPtrs) <= kPtrRecord, "pointer record too small");
    const BucketPtrs b = save_ptrs(c);
    std::memcpy(rec, &b, sizeof b);
}

void state_ptrs_load(Ctx* c, const void* rec) {
    BucketPtrs b;
    std::memcpy(&b, rec, sizeof b);
    load_ptrs(c, b);
}

// The graph form: keys (recording the movers) and the branch decision, then IF (radix) the
// radix sort, IF (previous order) the build from the previous order into the buffers the
// radix sort would leave its result in, then the common tail.
int bucket_append(Ctx* c, cudaGraph_t G, cudaGraphNode_t dep, cudaGraphNode_t* tail) {
    cudaStream_t s = c->stream;
    const cudaStreamCaptureMode mode = cudaStreamCaptureModeRelaxed;
    cudaGraph_t R = nullptr, I = nullptr, tmp = nullptr;
    cudaGraphConditionalHandle h_r = 0, h_i = 0;
    cudaGraphNode_t n_keys, n_r, n_i;
    int rc;
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_r, G, 0, cudaGraphCondAssignDefault));
    MPS_CUDA(c, cudaGraphConditionalHandleCreate(&h_i, G, 0, cudaGraphCondAssignDefault));
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                              mode));
    launch_keys(c, true, true);
    k_bucket_branch<<<1, 32, 0, s>>>(c->st, c->order_ok, c->mov_cap, h_r, h_i);
    c->launches += 1;
    n_keys = capture_tail(s);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    if (!n_keys) return MPS_EDEVICE;
    uint32_t* const k_new = c->key;   // the new keys in slot order
    uint32_t* const k_other = c->key_alt;
    int32_t* const v_other = c->perm_alt;
    // ---- IF: the radix sort
    if ((rc = add_cond(c, G, n_keys, h_r, cudaGraphCondTypeIf, &n_r, &R))) return rc;
    int64_t l = c->launches;
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, R, nullptr, nullptr, 0, mode));
    launch_radix(c);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    c->bucket_radix_launches = c->launches - l;
    c->launches = l;
    // ---- IF: from the previous order, into the buffers the radix sort leaves its result in
    // (through the other pair and a copy when that is where the new keys are)
    if ((rc = add_cond(c, G, n_r, h_i, cudaGraphCondTypeIf, &n_i, &I))) return rc;
    l = c->launches;
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, I, nullptr, nullptr, 0, mode));
    const size_t n = (size_t)c->n;
    if (c->key != k_new) {
        if ((rc = launch_from_previous(c, k_new, c->key, c->perm))) return rc;
    } else {
        if ((rc = launch_from_previous(c, k_new, k_other, v_other))) return rc;
        MPS_CUDA(c, cudaMemcpyAsync(c->key, k_other, n * sizeof(uint32_t),
                                    cudaMemcpyDeviceToDevice, s));
        MPS_CUDA(c, cudaMemcpyAsync(c->perm, v_other, n * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, s));
    }
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    c->bucket_inc_launches = c->launches - l;
    c->launches = l;
    // ---- the common tail
    MPS_CUDA(c, cudaStreamBeginCaptureToGraph(s, G, &n_i, nullptr, 1, mode));
    if ((rc = launch_table_rest(c))) return rc;
    *tail = capture_tail(s);
    MPS_CUDA(c, cudaStreamEndCapture(s, &tmp));
    if (!*tail) return MPS_EDEVICE;
    return MPS_OK;
}

void bucket_branch_count(Ctx* c, const DevStatus& st) {
    if (c->pending_branch < 0) return;
    const bool inc = c->pending_branch != 0 && st.n_mov <= (unsigned)c->mov_cap;
    c->launches += inc ? c->bucket_inc_launches : c->bucket_radix_launches;
    c->last_bucket_merged = inc ? 1 : 0;
    c->pending_branch = -1;
}

// the host's word for the next graph build: whether the slot order and cell table are those
// of the previous build with this grid
int bucket_order_word(Ctx* c) {
    const bool ok = c->order_valid && c->prm.bucket_sort == 0;
    MPS_CUDA(c, cudaMemsetAsync(c->order_ok, ok ? 1 : 0, sizeof(int32_t), c->stream));
    c->pending_branch = ok ? 1 : 0;
    return MPS_OK;
}

int bucket_build(Ctx* c, bool mutate) {
    if (!mutate || c->graphs_off || c->prm.step_graph == 2) return bucket_launches(c, mutate);
    BucketGraph* bg = nullptr;
    for (BucketGraph& g : c->bucket_graph)
        if (g.exec && g.pos == c->pos) bg = &g;
    if (!bg) {
        for (BucketGraph& g : c->bucket_graph)
            if (!g.exec) { bg = &g; break; }
        if (!bg) return bucket_launches(c, true);   // not expected: more than two parities
        const double4* start = c->pos;
        const BucketPtrs before = save_ptrs(c);
        const int64_t l0 = c->launches;
        MPS_CUDA(c, cudaStreamSynchronize(c->stream));
        cudaGraph_t g = nullptr;
        MPS_CUDA(c, cudaGraphCreate(&g, 0));
        cudaGraphNode_t tail = nullptr;
        int rc = bucket_append(c, g, nullptr, &tail);
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaGraphInstantiate(&bg->exec, g, 0);
        if (rc || e != cudaSuccess) {
            // the graph of a failed capture is left alone (the runtime may have dropped the
            // body it was capturing into)
            abort_capture(c);
            bg->exec = nullptr;
            c->graphs_off = true;
            load_ptrs(c, before);
            c->launches = l0;
            return rc ? rc : cuda_fail(c, e, "bucket graph instantiate");
        }
        bg->graph = g;
        bg->pos = start;
        bg->launches = c->launches - l0;
        BucketPtrs after = save_ptrs(c);
        static_assert(sizeof(BucketPtrs) <= sizeof(bg->after), "pointer record too small");
        std::memcpy(bg->after, &after, sizeof after);
        c->launches = l0;   // counted at the replay below
        load_ptrs(c, before);
    }
    if (int rc = bucket_order_word(c)) return rc;
    MPS_CUDA(c, cudaGraphLaunch(bg->exec, c->stream));
    BucketPtrs after;
    std::memcpy(&after, bg->after, sizeof after);
    load_ptrs(c, after);
    c->launches += bg->launches;
    c->order_valid = true;
    return MPS_OK;
}

void bucket_graphs_destroy(Ctx* c) {
    for (BucketGraph& g : c->bucket_graph) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        g = BucketGraph{};
    }
}

}  // namespace mps
