// Top-down backtracking with merging (Eq. 13-15) and reciprocal verification
// (Eq. 16).
//
// The tuple set starts as every position q of every existing top-level patch
// p with score C_L(p, q) (Sec. 3.3 "Merging correspondences").  One step maps
// a tuple (l, p, q, s) to its children (Eq. 13-14):
//   r = q + o_i (skipped outside the domain),  t = 2r + m_i (saved argmax),
//   child tuple (l-1, c_i, t, s + P_{l-1}(c_i, r)),
// and tuples equal in (l-1, c_i, t) are merged keeping the highest score.
//
// Only a small fraction of all (patch, position) pairs is ever reached (the
// merged frontier is typically 1-5% of a level's pooled map below the top), so
// the frontier is kept sparse: one open-addressing table per level keyed by
// (patch, position) with 64-bit slots (key+1) << 32 | score, merged by 64-bit
// atomicMax; the next step scans the table in slot order.  Where the keys
// patch * |domain| + position do not fit 32 bits (large or rotated images:
// the canvases of the invariant form), the slots are 16 bytes, {key + 1,
// score}: the key word is claimed by a 64-bit compare-and-swap and the score
// merged by atomicMax in its own word (the next step reads both after the
// kernel has ended).
// The active table size is derived on the device from the previous
// frontier's size, so nothing waits for the host.
//
// Path scores are exact: each term (a map value in [0, 1]) is rounded to the
// nearest multiple of 2^-28 and the terms are summed as unsigned 32-bit fixed
// point (L + 1 < 16 terms, so no overflow).  The sum is exact, so merging by
// maximum is independent of arrival order, and the fixed-point score orders
// like its value in the 32-bit score field of a slot.  It is rounded to FP32
// once, when a match is written.
//
// At the atomic level the tuples are reduced into two arrays of packed keys
// (score << 32 | ~index) with atomicMax:
//   BestAt(p)  per atomic patch (its own 4x4 cell of I), index = pixel of I';
//   BestAt'(c) per 4x4 cell of I',                      index = patch*16 + offset.
// A patch's best tuple is output iff it also wins its cell of I'.
#include "dm_internal.cuh"

#include <memory>

namespace {

constexpr int BT_BLOCK = 256;

// Path-score term: v in [0, 1] to unsigned fixed point, 28 fractional bits,
// round to nearest even (v * 2^28 is exact in FP32).
__device__ __forceinline__ unsigned int ps_term(float v) { return __float2uint_rn(__fmul_rn(v, 268435456.0f)); }
// Fixed-point score to FP32, rounded once.
__device__ __forceinline__ float ps_value(unsigned int s) { return __fmul_rn(__uint2float_rn(s), 0x1p-28f); }

struct BtArgs {
    DmGeom g;
    const unsigned char* valid[DM_MAXL + 1];
    const float* pooled[DM_MAXL];
    const unsigned char* amax[DM_MAXL];
    const float* top;
    unsigned long long* table[DM_MAXL + 1];
    unsigned int capmax[DM_MAXL + 1];
    unsigned long long* elist[DM_MAXL + 1];   // DM*: entry points found per level
    unsigned long long elcap[DM_MAXL + 1];
    unsigned long long* bestP;
    unsigned long long* bestQ;
    DmWsHeader* hdr;
    const int* proto_of;          // approximate form: level-0 map of atomic patch c is proto_of[c]; else null
    int n0_maps;                  // level-0 maps (entries of proto_of are clamped to [0, n0_maps))
    DmRect rect;                  // invariant form: rectification of the atomic tuples (RECT kernels only)
};

// Home slot of a key: keys are patch * |domain| + position, so 32 consecutive
// keys are 32 neighbouring positions of one patch on one row.  Such a block of
// keys keeps its 32 slots together (block index hashed, offset kept), and the
// expansion scans the table in slot order: a warp then handles neighbouring
// positions of one patch, whose children's map values and merge slots are
// neighbours too, so loads and atomics coalesce instead of scattering.
constexpr unsigned int HT_BLOCK_LOG2 = 5;           // 32 keys per block
constexpr unsigned long long HT_SLOTS_PER_PREV = 12;  // active slots per tuple of the previous frontier

__device__ __forceinline__ unsigned int ht_home(unsigned int key, unsigned int cap) {
    const unsigned int nblk = cap >> HT_BLOCK_LOG2;
    const unsigned int blk = (unsigned int)(((unsigned long long)((key >> HT_BLOCK_LOG2) * 2654435761u) * nblk) >> 32);
    return (blk << HT_BLOCK_LOG2) | (key & ((1u << HT_BLOCK_LOG2) - 1u));
}

// 64-bit keys: the block index is hashed from the 64-bit block number.
__device__ __forceinline__ unsigned int ht_home64(unsigned long long key, unsigned int cap) {
    const unsigned long long nblk = cap >> HT_BLOCK_LOG2;
    const unsigned long long hb = ((key >> HT_BLOCK_LOG2) * 0x9E3779B97F4A7C15ull) >> 32;
    const unsigned int blk = (unsigned int)((hb * nblk) >> 32);
    return (blk << HT_BLOCK_LOG2) | (unsigned int)(key & ((1u << HT_BLOCK_LOG2) - 1u));
}

// Merge (key, score) into a level table of 16-byte slots; returns 1 if the key is new.
__device__ __forceinline__ int ht_insert64(const BtArgs& a, int lvl, unsigned int cap, unsigned long long key, unsigned int sb) {
    ulonglong2* tab = reinterpret_cast<ulonglong2*>(a.table[lvl]);
    const unsigned long long kw = key + 1ull;
    unsigned int h = ht_home64(key, cap);
    for (unsigned int probe = 0; probe < cap; probe++) {
        unsigned long long cur = __ldcg(&tab[h].x);
        if (cur == 0ull) {
            const unsigned long long prev = atomicCAS(&tab[h].x, 0ull, kw);
            if (prev == 0ull) {
                atomicMax(&tab[h].y, (unsigned long long)sb);
                return 1;
            }
            cur = prev;
        }
        if (cur == kw) {
            if (__ldcg(&tab[h].y) < (unsigned long long)sb) atomicMax(&tab[h].y, (unsigned long long)sb);
            return 0;
        }
        h = (h + 1u == cap) ? 0u : h + 1u;
    }
    atomicOr(&a.hdr->status, DM_DEV_FRONTIER_OVERFLOW);
    return 0;
}

// Merge (key, score) into the level-`lvl` table; returns 1 if the key is new.
// (New keys are counted by the caller and added to the level's count once per
// block: a shared counter bumped by every warp serialised the whole pass.)
__device__ __forceinline__ int ht_insert(const BtArgs& a, int lvl, unsigned int cap, unsigned int key, unsigned int sb) {
    unsigned long long* tab = a.table[lvl];
    const unsigned long long packed = ((unsigned long long)(key + 1u) << 32) | sb;
    unsigned int h = ht_home(key, cap);
    for (unsigned int probe = 0; probe < cap; probe++) {
        unsigned long long cur = __ldcg(tab + h);
        if (cur == 0ull) {
            unsigned long long prev = atomicCAS(tab + h, 0ull, packed);
            if (prev == 0ull) return 1;
            cur = prev;
        }
        if ((unsigned int)(cur >> 32) == key + 1u) {
            if ((unsigned int)cur < sb) atomicMax(tab + h, packed);
            return 0;
        }
        h = (h + 1u == cap) ? 0u : h + 1u;
    }
    atomicOr(&a.hdr->status, DM_DEV_FRONTIER_OVERFLOW);
    return 0;
}

__device__ __forceinline__ void leaf_update(const BtArgs& a, int c, int tx, int ty, unsigned int s) {
    const DmGeom& g = a.g;
    const unsigned long long sb = (unsigned long long)s << 32;
    unsigned int tidx = (unsigned int)(ty * g.W2 + tx);
    unsigned long long kp = sb | (0xffffffffu - tidx);
    if (__ldcg(a.bestP + c) < kp) atomicMax(a.bestP + c, kp);
    int CW = (g.W2 + 3) >> 2;
    int cell = (ty >> 2) * CW + (tx >> 2);
    unsigned int qidx = (unsigned int)c * 16u + (unsigned int)((ty & 3) * 4 + (tx & 3));
    unsigned long long kq = sb | (0xffffffffu - qidx);
    if (__ldcg(a.bestQ + cell) < kq) atomicMax(a.bestQ + cell, kq);
}

// Nearest pixel index floor(x + 1/2), clamped to [0, n).
__device__ __forceinline__ int round_px(float x, int n) {
    const float f = floorf(__fadd_rn(x, 0.5f));
    if (!(f > 0.0f)) return 0;
    return f >= (float)(n - 1) ? n - 1 : (int)f;
}

// Invariant form (Algorithm 2): the atomic tuple (c, t, s) of one transform
// rectified to the input pair -- the centre of warped patch c taken back to
// image 1 and rounded to a pixel, whose atomic patch (4x4 cell) becomes the
// tuple's patch; canvas pixel t taken back to image 2 and rounded -- and
// reduced into the input pair's BestAt / BestAt' with the same keys as above.
__device__ __forceinline__ void leaf_update_rect(const BtArgs& a, int c, int tx, int ty, unsigned int s) {
    const DmRect& r = a.rect;
    const int gx = a.g.P0x;
    float x1, y1, x2, y2;
    dm_to_source(r.t1, (float)(4 * (c % gx) + 2), (float)(4 * (c / gx) + 2), x1, y1);
    dm_to_source(r.t2, (float)tx, (float)ty, x2, y2);
    const int X1 = round_px(x1, r.W1), Y1 = round_px(y1, r.H1);
    const int X2 = round_px(x2, r.W2), Y2 = round_px(y2, r.H2);
    const int C1 = min(Y1 >> 2, r.P0y - 1) * r.P0x + min(X1 >> 2, r.P0x - 1);
    const unsigned long long sb = (unsigned long long)s << 32;
    const unsigned long long kp = sb | (0xffffffffu - (unsigned int)(Y2 * r.W2 + X2));
    if (__ldcg(r.bestP + C1) < kp) atomicMax(r.bestP + C1, kp);
    const int cell = (Y2 >> 2) * ((r.W2 + 3) >> 2) + (X2 >> 2);
    const unsigned int qidx = (unsigned int)C1 * 16u + (unsigned int)((Y2 & 3) * 4 + (X2 & 3));
    const unsigned long long kq = sb | (0xffffffffu - qidx);
    if (__ldcg(r.bestQ + cell) < kq) atomicMax(r.bestQ + cell, kq);
}

// Children of tuple (l, p, q, s); returns the number of atomic arrivals.
// The (up to 4) children's pooled values and argmax codes are loaded first,
// all independent, so their memory latencies overlap; the merges follow.
// Variants of the expansion: the new form, the invariant form's rectified
// leaves, and DM* (start score carried down unchanged, the end value added at
// the leaf).
constexpr int BT_EXACT = 0, BT_RECT = 1, BT_STAR = 2;

template <int MODE, bool K64>
__device__ __forceinline__ int expand(const BtArgs& a, int l, unsigned int cap_next, int p, int qx, int qy, unsigned int s) {
    const DmGeom& g = a.g;
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);    // pooled map P_{l-1} lives on domain l
    const int ix = p % g.Lx, iy = p / g.Lx;
    int cc[4], rxs[4], rys[4];
    float val[4];
    int code[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        cc[i] = -1;
        int c = dm_child(g, l, ix, iy, i);
        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        int rx = qx + ox, ry = qy + oy;
        if (c >= 0 && rx >= 0 && ry >= 0 && rx < mw && ry < mh && a.valid[l - 1][c]) {
            cc[i] = c;
            rxs[i] = rx;
            rys[i] = ry;
            const int cm = (l == 1 && a.proto_of) ? min(max(__ldg(a.proto_of + c), 0), a.n0_maps - 1) : c;   // its map
            long long ro = ((long long)cm * mh + ry) * pitch + rx;
            code[i] = a.amax[l - 1][ro];
            val[i] = a.pooled[l - 1][ro];
        }
    }
    int arrivals = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        // a code above 8 never comes from the pooling (first in-domain maximum of
        // 9); it can only be left by a level kernel whose bounded wait gave up
        // (status DM_DEV_TIMEOUT): skipping it keeps every position in its domain
        if (cc[i] < 0 || code[i] > 8) continue;
        const int rx = rxs[i], ry = rys[i];
        const int tx = 2 * rx + code[i] % 3 - 1, ty = 2 * ry + code[i] / 3 - 1;
        const unsigned int s2 = (MODE == BT_STAR && l - 1 >= 1) ? s : s + ps_term(val[i]);
        if (l - 1 >= 1) {
            if constexpr (K64) {
                const unsigned long long key = (unsigned long long)cc[i] * (unsigned long long)g.dsize(l - 1) +
                                               (unsigned long long)(ty * g.dw[l - 1] + tx);
                arrivals += ht_insert64(a, l - 1, cap_next, key, s2);
            } else {
                const unsigned int key = (unsigned int)cc[i] * (unsigned int)g.dsize(l - 1) + (unsigned int)(ty * g.dw[l - 1] + tx);
                arrivals += ht_insert(a, l - 1, cap_next, key, s2);
            }
        } else {
            if constexpr (MODE == BT_RECT) leaf_update_rect(a, cc[i], tx, ty, s2);
            else leaf_update(a, cc[i], tx, ty, s2);
            arrivals++;
        }
    }
    return arrivals;
}

// Add the block's count to count[lvl]: a warp sum, a shared-memory sum, one
// global atomic per block.  Every thread of the block reaches this point.
__device__ __forceinline__ void add_count(const BtArgs& a, int lvl, int n) {
    __shared__ unsigned int blk;
    if (threadIdx.x == 0) blk = 0u;
    __syncthreads();
    const int tot = __reduce_add_sync(0xffffffffu, n);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(&blk, (unsigned int)tot);
    __syncthreads();
    if (threadIdx.x == 0 && blk) atomicAdd(&a.hdr->count[lvl], blk);
}

// Clear the active part of the level-`lvl` table.  Active size: 12x the
// previous frontier (4 children per tuple: load <= 1/3, few collisions
// between the 32-slot key blocks), a multiple of 32 within [64, capmax].
template <bool K64 = false>
__device__ __forceinline__ void clear_table(const BtArgs& a, int lvl, unsigned long long cap) {
    if (cap < 64ull) cap = 64ull;
    const unsigned long long cmax = (unsigned long long)a.capmax[lvl] & ~31ull;
    if (cap > cmax) cap = cmax;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.hdr->cap[lvl] = (unsigned int)cap;
    const unsigned long long words = K64 ? 2ull * cap : cap;     // 16-byte slots hold two words
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (unsigned long long)gridDim.x * blockDim.x)
        a.table[lvl][i] = 0ull;
}

// DM*: the level-`lvl` table also receives that level's entry points (counted
// before the backtracking starts); 3 slots per entry (load <= 1/3, like the
// children's 12 per tuple of 4 children).
__global__ void k_star_prepare(BtArgs a, int lvl) {
    const unsigned long long n_prev = lvl == a.g.L ? 0ull : a.hdr->count[lvl + 1];
    clear_table(a, lvl, (n_prev * HT_SLOTS_PER_PREV + 3ull * a.hdr->entries[lvl] + 31ull) & ~31ull);
}

template <bool K64>
__device__ __forceinline__ void bt_prepare_body(const BtArgs& a, int lvl, long long n_top) {
    const unsigned long long n_prev = (lvl + 1 == a.g.L) ? (unsigned long long)n_top : a.hdr->count[lvl + 1];
    clear_table<K64>(a, lvl, (n_prev * HT_SLOTS_PER_PREV + 31ull) & ~31ull);
}

template <bool K64>
__global__ void k_bt_prepare(BtArgs a, int lvl, long long n_top) { bt_prepare_body<K64>(a, lvl, n_top); }

// Expansion of the top level: every position of every existing top patch.
template <int MODE, bool K64>
__device__ __forceinline__ void bt_expand_top_body(const BtArgs& a) {
    const DmGeom& g = a.g;
    const int L = g.L;
    const long long ds = g.dsize(L);
    const long long n = (long long)g.npatch(L) * ds;
    const unsigned int cap_next = (L - 1 >= 1) ? a.hdr->cap[L - 1] : 0u;
    int arrivals = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e - threadIdx.x < n;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < n) {
            int p = (int)(e / ds);
            int q = (int)(e % ds);
            if (a.valid[L][p]) {
                if (q == 0) atomicAdd(&a.hdr->count[L], (unsigned int)ds);
                arrivals += expand<MODE, K64>(a, L, cap_next, p, q % g.dw[L], q / g.dw[L], ps_term(a.top[e]));
            }
        }
    }
    add_count(a, L - 1, arrivals);
}

template <int MODE, bool K64>
__global__ void k_bt_expand_top(BtArgs a) { bt_expand_top_body<MODE, K64>(a); }

// Expansion of level l < L: the merged tuples of level l, read by scanning the
// active part of its table in slot order.  Each warp packs the occupied slots
// it reads into a queue in shared memory and expands them 32 at a time, so its
// lanes stay busy while the slot order (neighbouring positions of one patch
// together) is kept.
template <int MODE, bool K64>
__device__ __forceinline__ void bt_expand_body(const BtArgs& a, int l) {
    // queued slots: the packed slot (32-bit keys), or key + 1 and score
    __shared__ unsigned long long queue[BT_BLOCK / 32][64];
    __shared__ unsigned int qscore[K64 ? BT_BLOCK / 32 : 1][64];
    const DmGeom& g = a.g;
    const unsigned int cap = a.hdr->cap[l];
    const unsigned int cap_next = (l - 1 >= 1) ? a.hdr->cap[l - 1] : 0u;
    const unsigned int ds = (unsigned int)g.dsize(l);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long* q = queue[warp];
    unsigned int* qs = qscore[K64 ? warp : 0];
    int qn = 0;                                          // warp-uniform queue length
    int arrivals = 0;
    auto run = [&](unsigned long long v, unsigned int sc64) {
        int p, t;
        unsigned int sc;
        if constexpr (K64) {
            const unsigned long long key = v - 1ull;
            p = (int)(key / ds);
            t = (int)(key - (unsigned long long)p * ds);
            sc = sc64;
        } else {
            const unsigned int key = (unsigned int)(v >> 32) - 1u;
            sc = (unsigned int)v;
            p = (int)(key / ds);
            t = (int)(key % ds);
        }
        arrivals += expand<MODE, K64>(a, l, cap_next, p, t % g.dw[l], t / g.dw[l], sc);
    };
    for (unsigned int i0 = blockIdx.x * blockDim.x; i0 < cap; i0 += gridDim.x * blockDim.x) {
        const unsigned int i = i0 + threadIdx.x;
        unsigned long long v = 0ull;
        unsigned int sc = 0u;
        if constexpr (K64) {
            if (i < cap) {
                const ulonglong2 w = __ldcg(reinterpret_cast<const ulonglong2*>(a.table[l]) + i);
                v = w.x;
                sc = (unsigned int)w.y;
            }
        } else {
            v = i < cap ? __ldcg(a.table[l] + i) : 0ull;
        }
        const unsigned int occ = __ballot_sync(0xffffffffu, v != 0ull);
        if (v != 0ull) {
            const int at = qn + __popc(occ & ((1u << lane) - 1u));
            q[at] = v;
            if constexpr (K64) qs[at] = sc;
        }
        qn += __popc(occ);
        __syncwarp();
        if (qn >= 32) {
            const unsigned long long w = q[lane];
            const unsigned int ws = K64 ? qs[lane] : 0u;
            const unsigned long long rest = lane + 32 < qn ? q[lane + 32] : 0ull;
            const unsigned int rests = (K64 && lane + 32 < qn) ? qs[lane + 32] : 0u;
            __syncwarp();
            if (lane + 32 < qn) {
                q[lane] = rest;
                if constexpr (K64) qs[lane] = rests;
            }
            qn -= 32;
            __syncwarp();
            run(w, ws);
        }
    }
    if (lane < qn) run(q[lane], K64 ? qs[lane] : 0u);
    add_count(a, l - 1, arrivals);
}

template <int MODE, bool K64>
__global__ void k_bt_expand(BtArgs a, int l) { bt_expand_body<MODE, K64>(a, l); }

// Reciprocal verification and compaction in atomic-patch order (one block).
__device__ __forceinline__ void reciprocal_body(const BtArgs& a, dm_match_t* __restrict__ out, int capacity,
                                                int* __restrict__ d_count) {
    const DmGeom& g = a.g;
    const int n0 = g.npatch(0);
    const int CW = (g.W2 + 3) >> 2;
    const int chunk = (n0 + blockDim.x - 1) / blockDim.x;
    const int p0 = threadIdx.x * chunk;
    const int p1 = min(n0, p0 + chunk);
    __shared__ int warp_sums[32];
    __shared__ int total;

    auto survives = [&](int p, int& tx, int& ty, float& s) -> bool {
        unsigned long long kp = a.bestP[p];
        if (kp == 0ull) return false;
        unsigned int tidx = 0xffffffffu - (unsigned int)kp;
        tx = (int)(tidx % (unsigned int)g.W2);
        ty = (int)(tidx / (unsigned int)g.W2);
        int cell = (ty >> 2) * CW + (tx >> 2);
        unsigned long long kq = a.bestQ[cell];
        unsigned int qidx = 0xffffffffu - (unsigned int)kq;
        s = ps_value((unsigned int)(kp >> 32));
        return (kq >> 32) == (kp >> 32) && qidx == (unsigned int)p * 16u + (unsigned int)((ty & 3) * 4 + (tx & 3));
    };

    int mine = 0;
    for (int p = p0; p < p1; p++) {
        int tx, ty;
        float s;
        mine += survives(p, tx, ty, s) ? 1 : 0;
    }
    // block exclusive scan of `mine`
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_sums[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += v;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == 31) total = wi;
    }
    __syncthreads();
    int pos = warp_sums[warp] + incl - mine;
    for (int p = p0; p < p1; p++) {
        int tx, ty;
        float s;
        if (survives(p, tx, ty, s)) {
            if (pos < capacity) {
                dm_match_t m;
                m.x1 = (float)(4 * (p % g.P0x) + 2);
                m.y1 = (float)(4 * (p / g.P0x) + 2);
                m.x2 = (float)tx;
                m.y2 = (float)ty;
                m.score = s;
                out[pos] = m;
            }
            pos++;
        }
    }
    if (threadIdx.x == 0) {
        *d_count = total;
        if (total > capacity) atomicOr(&a.hdr->status, DM_DEV_OUTPUT_OVERFLOW);
    }
}

__global__ void __launch_bounds__(1024) k_reciprocal(BtArgs a, dm_match_t* __restrict__ out, int capacity,
                                                     int* __restrict__ d_count) {
    reciprocal_body(a, out, capacity, d_count);
}

// DM* entry points at level l (1..L): the local maxima of the maps C_l(p, .)
// of the existing patches.  q is one iff A(q) > 0 and, over its in-domain
// 8-neighbours r, A(q) > A(r) for r before q in row-major order and
// A(q) >= A(r) for r after it, A being the unrectified average of the level
// pass (same arithmetic, hence the same order as C_l = A^lambda).
//
// One warp streams down a strip of 30 columns of one patch's map (lane j
// holds column x0 - 1 + j, so lanes 0 and 31 are the halo), ST_ROWS rows per
// work item: each step forms one new row of averages (4 coalesced child loads
// per lane) and tests the row above it against the three rows held in
// registers, horizontal neighbours by shuffles.  No shared memory and no
// block barrier.  Each entry (l, p, q) with score C_l(p, q) is appended to
// the level's list (hdr->entries[l] counts them; the merge tables are sized
// from the counts before anything is inserted).
constexpr int ST_COLS = 30, ST_ROWS = 32;

// Each warp gathers the entry points it finds in a shared-memory buffer of
// STAR_BUF and appends a full buffer to the level's list with one global
// atomic for the whole buffer (instead of one per group of maxima found, all
// on one counter), so the list stays dense.
constexpr unsigned int STAR_BUF = 256;

__device__ __forceinline__ void star_flush(const BtArgs& a, int l, const unsigned long long* buf, unsigned int n, int lane) {
    __syncwarp();
    unsigned int base = 0u;
    if (lane == 0 && n) base = atomicAdd(&a.hdr->entries[l], n);
    base = __shfl_sync(0xffffffffu, base, 0);
    bool over = false;
    for (unsigned int j = (unsigned int)lane; j < n; j += 32u) {
        if (base + j < a.elcap[l]) a.elist[l][base + j] = buf[j];
        else over = true;
    }
    if (over) atomicOr(&a.hdr->status, DM_DEV_FRONTIER_OVERFLOW);
    __syncwarp();
}

template <bool COMP>
__global__ void __launch_bounds__(256) k_star_entries(BtArgs a, int l, float lam, long long n_items) {
    const DmGeom& g = a.g;
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);
    const int strips = (mw + ST_COLS - 1) / ST_COLS, tiles = strips * ((mh + ST_ROWS - 1) / ST_ROWS);
    const unsigned int ds = (unsigned int)g.dsize(l);
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    __shared__ unsigned long long sbuf[8][STAR_BUF];    // (blocks of 8 warps)
    unsigned long long* buf = sbuf[threadIdx.x >> 5];
    unsigned int nbuf = 0u;                             // entries in this warp's buffer
    for (long long it = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); it < n_items; it += warps) {
        const int p = (int)(it / tiles), t = (int)(it % tiles);
        if (!a.valid[l][p]) continue;                  // the same for the whole warp
        Kids k;
        load_kids(g, l, p, a.valid[l - 1], a.pooled[l - 1], k, l == 1 ? a.proto_of : nullptr, a.n0_maps);
        const int x = (t % strips) * ST_COLS - 1 + lane;
        const int y0 = (t / strips) * ST_ROWS;
        const int y1 = min(y0 + ST_ROWS, mh);          // rows y0 .. y1-1 are tested
        const bool col_in = x >= 0 && x < mw;
        auto avg = [&](int y) -> float {
            return (col_in && y >= 0 && y < mh) ? child_mean<COMP>(k, x, y, mw, mh, pitch) : -INFINITY;
        };
        float up = avg(y0 - 1), mid = avg(y0);
        for (int y = y0; y < y1; y++) {
            const float dn = avg(y + 1);
            const float ul = __shfl_up_sync(0xffffffffu, up, 1), ur = __shfl_down_sync(0xffffffffu, up, 1);
            const float ml = __shfl_up_sync(0xffffffffu, mid, 1), mr = __shfl_down_sync(0xffffffffu, mid, 1);
            const float dl = __shfl_up_sync(0xffffffffu, dn, 1), dr = __shfl_down_sync(0xffffffffu, dn, 1);
            const float v = mid;
            const bool m = lane >= 1 && lane <= ST_COLS && col_in && v > 0.0f && v > ul && v > up && v > ur && v > ml &&
                           v >= mr && v >= dl && v >= dn && v >= dr;
            const unsigned int found = __ballot_sync(0xffffffffu, m);
            if (found) {
                const unsigned int cnt = (unsigned int)__popc(found);
                if (nbuf + cnt > STAR_BUF) {
                    star_flush(a, l, buf, nbuf, lane);
                    nbuf = 0u;
                }
                if (m) {
                    const unsigned int key = (unsigned int)p * ds + (unsigned int)(y * mw + x);
                    buf[nbuf + (unsigned int)__popc(found & ((1u << lane) - 1u))] =
                        ((unsigned long long)key << 32) | ps_term(dm_powf(v, lam));
                }
                nbuf += cnt;
            }
            up = mid;
            mid = dn;
        }
    }
    star_flush(a, l, buf, nbuf, lane);
}

// DM*: the level-l entry points merged into the level-l table.
__global__ void k_star_insert(BtArgs a, int l) {
    const unsigned int cap = a.hdr->cap[l];
    const unsigned long long n = min((unsigned long long)a.hdr->entries[l], a.elcap[l]);
    int fresh = 0;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long e = a.elist[l][i];
        fresh += ht_insert(a, l, cap, (unsigned int)(e >> 32), (unsigned int)e);
    }
    add_count(a, l, fresh);
}

template <int MODE, bool K64>
void launch_steps_k(const BtArgs& a, int grid, cudaStream_t st) {
    const DmGeom& g = a.g;
    const long long n_top = (long long)g.npatch(g.L) * g.dsize(g.L);
    for (int l = g.L; l >= 1; l--) {
        if (l - 1 >= 1) k_bt_prepare<K64><<<grid, BT_BLOCK, 0, st>>>(a, l - 1, n_top);
        if (l == g.L) {
            long long nb = (n_top + BT_BLOCK - 1) / BT_BLOCK;
            k_bt_expand_top<MODE, K64><<<(unsigned)(nb < grid ? nb : grid), BT_BLOCK, 0, st>>>(a);
        } else {
            k_bt_expand<MODE, K64><<<grid, BT_BLOCK, 0, st>>>(a, l);
        }
    }
}

template <int MODE>
void launch_steps(const BtArgs& a, int grid, cudaStream_t st) {
    if (a.g.key64) launch_steps_k<MODE, true>(a, grid, st);
    else launch_steps_k<MODE, false>(a, grid, st);
}

}  // namespace

namespace {

// Arguments of one pair's backtracking over workspace ws (layout bl).
BtArgs make_bt_args(const DmGeom& g, const dm_pyramid& py, const DmBtLayout& bl, char* ws) {
    BtArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.proto_of = py.proto_of;
    a.n0_maps = py.n0_maps;
    for (int l = 0; l <= g.L; l++) a.valid[l] = py.valid[l];
    for (int l = 0; l < g.L; l++) {
        a.pooled[l] = py.pooled[l];
        a.amax[l] = py.amax[l];
    }
    a.top = py.top;
    for (int l = 1; l < g.L; l++) {
        a.table[l] = reinterpret_cast<unsigned long long*>(ws + bl.table[l]);
        a.capmax[l] = (unsigned int)bl.cap[l];
    }
    a.bestP = reinterpret_cast<unsigned long long*>(ws + bl.bestP);
    a.bestQ = reinterpret_cast<unsigned long long*>(ws + bl.bestQ);
    a.hdr = reinterpret_cast<DmWsHeader*>(ws + bl.header);
    return a;
}

// Clear the backtracking part of the header (status word, counts, table
// sizes; pyr_status belongs to the pyramid step that ran before) and, unless
// the tuples go to another pair's keys (rect), the BestAt / BestAt' keys.
cudaError_t clear_bt(const BtArgs& a, bool keys, cudaStream_t st) {
    const DmGeom& g = a.g;
    cudaError_t e;
    if ((e = cudaMemsetAsync(&a.hdr->status, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.hdr->count, 0, sizeof(a.hdr->count) + sizeof(a.hdr->cap), st)) != cudaSuccess) return e;
    if (keys) {
        if ((e = cudaMemsetAsync(a.bestP, 0, sizeof(unsigned long long) * g.npatch(0), st)) != cudaSuccess) return e;
        size_t ncell = (size_t)((g.W2 + 3) / 4) * ((g.H2 + 3) / 4);
        if ((e = cudaMemsetAsync(a.bestQ, 0, sizeof(unsigned long long) * ncell, st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int sm_count() {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    return nsm;
}

// Cross-pair form: the pairs of a wave of the batched form in one launch per
// step, pair blockIdx.y (blockIdx.x for the reciprocal step), its arguments in
// the kernel parameters (a captured graph replays them as they were).  Step s
// of the backtracking works on level lvl[j] = L_j - s of pair j.
struct BtBatch {
    BtArgs a[DM_BATCH_MAX];
    int lvl[DM_BATCH_MAX];
    dm_match_t* out[DM_BATCH_MAX];
    int capacity[DM_BATCH_MAX];
    int* count[DM_BATCH_MAX];
    int n;
};
static_assert(sizeof(BtBatch) < 32000, "the kernel parameters of a wave must stay below the 32 KB limit");

template <bool K64>
__global__ void k_bt_prepare_b(const __grid_constant__ BtBatch B) {
    const BtArgs& a = B.a[blockIdx.y];
    bt_prepare_body<K64>(a, B.lvl[blockIdx.y] - 1, (long long)a.g.npatch(a.g.L) * a.g.dsize(a.g.L));
}

template <bool K64>
__global__ void k_bt_expand_top_b(const __grid_constant__ BtBatch B) {
    bt_expand_top_body<BT_EXACT, K64>(B.a[blockIdx.y]);
}

template <bool K64>
__global__ void k_bt_expand_b(const __grid_constant__ BtBatch B) {
    bt_expand_body<BT_EXACT, K64>(B.a[blockIdx.y], B.lvl[blockIdx.y]);
}

__global__ void __launch_bounds__(1024) k_reciprocal_b(const __grid_constant__ BtBatch B) {
    reciprocal_body(B.a[blockIdx.x], B.out[blockIdx.x], B.capacity[blockIdx.x], B.count[blockIdx.x]);
}

}  // namespace

cudaError_t dm_launch_backtrack(const DmGeom& g, const dm_pyramid& py, const DmBtLayout& bl, char* ws,
                                dm_match_t* out, int capacity, int* d_count, cudaStream_t st, const DmRect* rect) {
    BtArgs a = make_bt_args(g, py, bl, ws);
    if (rect) a.rect = *rect;
    cudaError_t e = clear_bt(a, !rect, st);
    if (e != cudaSuccess) return e;
    const int grid = sm_count() * (py.tune.bt_mult > 0 ? py.tune.bt_mult : 8);
    if (rect) {
        launch_steps<BT_RECT>(a, grid, st);
        dm_count_launches(2 * g.L - 1);
        return cudaGetLastError();
    }
    launch_steps<BT_EXACT>(a, grid, st);
    k_reciprocal<<<1, 1024, 0, st>>>(a, out, capacity, d_count);
    dm_count_launches(2 * g.L);
    return cudaGetLastError();
}

cudaError_t dm_launch_backtrack_star(const DmGeom& g, const dm_pyramid& py, const DmBtLayout& bl, char* ws, float lam,
                                     dm_match_t* out, int capacity, int* d_count, cudaStream_t st) {
    BtArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.proto_of = py.proto_of;
    a.n0_maps = py.n0_maps;
    for (int l = 0; l <= g.L; l++) a.valid[l] = py.valid[l];
    for (int l = 0; l < g.L; l++) {
        a.pooled[l] = py.pooled[l];
        a.amax[l] = py.amax[l];
    }
    a.top = py.top;
    for (int l = 1; l <= g.L; l++) {
        a.table[l] = reinterpret_cast<unsigned long long*>(ws + bl.table[l]);
        a.capmax[l] = (unsigned int)bl.cap[l];
        a.elist[l] = reinterpret_cast<unsigned long long*>(ws + bl.elist[l]);
        a.elcap[l] = bl.elcap[l];
    }
    a.bestP = reinterpret_cast<unsigned long long*>(ws + bl.bestP);
    a.bestQ = reinterpret_cast<unsigned long long*>(ws + bl.bestQ);
    a.hdr = reinterpret_cast<DmWsHeader*>(ws + bl.header);

    cudaError_t e;
    if ((e = cudaMemsetAsync(&a.hdr->status, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.hdr->count, 0, sizeof(a.hdr->count) + sizeof(a.hdr->cap) + sizeof(a.hdr->entries), st)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(a.bestP, 0, sizeof(unsigned long long) * g.npatch(0), st)) != cudaSuccess) return e;
    const size_t ncell = (size_t)((g.W2 + 3) / 4) * ((g.H2 + 3) / 4);
    if ((e = cudaMemsetAsync(a.bestQ, 0, sizeof(unsigned long long) * ncell, st)) != cudaSuccess) return e;

    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int grid = nsm * (py.tune.bt_mult > 0 ? py.tune.bt_mult : 8);
    auto items = [&](int l) -> long long {
        return (long long)g.npatch(l) * ((g.dw[l] + ST_COLS - 1) / ST_COLS) * ((g.dh[l] + ST_ROWS - 1) / ST_ROWS);
    };
    for (int l = 1; l <= g.L; l++) {
        const long long n = items(l);                   // one warp per item, 8 per CTA
        const long long nb = (n + 7) / 8;
        const unsigned gb = (unsigned)(nb < 8LL * nsm ? nb : 8LL * nsm);
        if (py.compensated) k_star_entries<true><<<gb, 256, 0, st>>>(a, l, lam, n);
        else k_star_entries<false><<<gb, 256, 0, st>>>(a, l, lam, n);
    }
    k_star_prepare<<<grid, BT_BLOCK, 0, st>>>(a, g.L);
    k_star_insert<<<grid, BT_BLOCK, 0, st>>>(a, g.L);
    for (int l = g.L; l >= 1; l--) {
        if (l - 1 >= 1) {
            k_star_prepare<<<grid, BT_BLOCK, 0, st>>>(a, l - 1);
            k_star_insert<<<grid, BT_BLOCK, 0, st>>>(a, l - 1);
        }
        k_bt_expand<BT_STAR, false><<<grid, BT_BLOCK, 0, st>>>(a, l);
    }
    k_reciprocal<<<1, 1024, 0, st>>>(a, out, capacity, d_count);
    dm_count_launches(4 * g.L + 1);
    return cudaGetLastError();
}

cudaError_t dm_launch_reciprocal(const DmGeom& g, unsigned long long* bestP, unsigned long long* bestQ, DmWsHeader* hdr,
                                 dm_match_t* out, int capacity, int* d_count, cudaStream_t st) {
    BtArgs a;
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.bestP = bestP;
    a.bestQ = bestQ;
    a.hdr = hdr;
    k_reciprocal<<<1, 1024, 0, st>>>(a, out, capacity, d_count);
    dm_count_launches(1);
    return cudaGetLastError();
}

// Backtracking and reciprocal verification of the n <= DM_BATCH_MAX pairs of
// a wave (pyramids computed): per step of the descent one launch per kernel
// (and merge-key width in use) for every pair still descending, then one
// reciprocal launch for all.
cudaError_t dm_launch_backtrack_batch(const dm_pyramid* const* pys, const DmBtLayout* const* bls, char* const* wss,
                                      dm_match_t* const* outs, const int* caps, int* const* counts, int n, cudaStream_t st) {
    if (n < 1 || n > DM_BATCH_MAX) return cudaErrorInvalidValue;
    // (host staging of the parameter blocks, ~20 KB each; a launch copies them)
    std::unique_ptr<BtBatch> all_p(new BtBatch), sub_p(new BtBatch), part_p(new BtBatch);
    BtBatch& all = *all_p;
    memset(&all, 0, sizeof(all));
    all.n = n;
    int Lmax = 0, mult = 8;
    cudaError_t e;
    for (int j = 0; j < n; j++) {
        all.a[j] = make_bt_args(pys[j]->g, *pys[j], *bls[j], wss[j]);
        all.out[j] = outs[j];
        all.capacity[j] = caps[j];
        all.count[j] = counts[j];
        if ((e = clear_bt(all.a[j], true, st)) != cudaSuccess) return e;
        Lmax = max(Lmax, pys[j]->g.L);
        if (pys[j]->tune.bt_mult > 0) mult = pys[j]->tune.bt_mult;
    }
    const int nsm = sm_count();
    // blocks per pair: the single-pair grid shared by the wave, at least one per SM
    const int per = max(nsm, nsm * mult / n);
    long long launches = 0;
    BtBatch& sub = *sub_p;
    for (int step = 0; step < Lmax; step++) {
        for (int k64 = 0; k64 < 2; k64++) {
            // the pairs still descending at this step with this key width
            memset(&sub, 0, sizeof(sub));
            long long top_max = 0;
            for (int j = 0; j < n; j++) {
                const DmGeom& g = pys[j]->g;
                if (step >= g.L || g.key64 != k64) continue;
                sub.a[sub.n] = all.a[j];
                sub.lvl[sub.n] = g.L - step;
                sub.n++;
                top_max = max(top_max, (long long)g.npatch(g.L) * g.dsize(g.L));
            }
            if (sub.n == 0) continue;
            // tables of the next level down (for the pairs that have one)
            BtBatch& b = sub;
            int with_next = 0;
            for (int j = 0; j < b.n; j++) with_next += b.lvl[j] - 1 >= 1;
            if (with_next == b.n) {
                if (k64) k_bt_prepare_b<true><<<dim3(per, b.n), BT_BLOCK, 0, st>>>(b);
                else k_bt_prepare_b<false><<<dim3(per, b.n), BT_BLOCK, 0, st>>>(b);
                launches++;
            } else if (with_next > 0) {
                // (pairs at level 1 have no table below: launched without them)
                BtBatch& part = *part_p;
                memset(&part, 0, sizeof(part));
                for (int j = 0; j < b.n; j++)
                    if (b.lvl[j] - 1 >= 1) {
                        part.a[part.n] = b.a[j];
                        part.lvl[part.n] = b.lvl[j];
                        part.n++;
                    }
                if (k64) k_bt_prepare_b<true><<<dim3(per, part.n), BT_BLOCK, 0, st>>>(part);
                else k_bt_prepare_b<false><<<dim3(per, part.n), BT_BLOCK, 0, st>>>(part);
                launches++;
            }
            if (step == 0) {
                const long long nb = (top_max + BT_BLOCK - 1) / BT_BLOCK;
                const unsigned gx = (unsigned)(nb < per ? nb : per);
                if (k64) k_bt_expand_top_b<true><<<dim3(gx, b.n), BT_BLOCK, 0, st>>>(b);
                else k_bt_expand_top_b<false><<<dim3(gx, b.n), BT_BLOCK, 0, st>>>(b);
            } else {
                if (k64) k_bt_expand_b<true><<<dim3(per, b.n), BT_BLOCK, 0, st>>>(b);
                else k_bt_expand_b<false><<<dim3(per, b.n), BT_BLOCK, 0, st>>>(b);
            }
            launches++;
        }
    }
    k_reciprocal_b<<<n, 1024, 0, st>>>(all);
    dm_count_launches(launches + 1);
    return cudaGetLastError();
}
