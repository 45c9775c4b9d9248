// Internal declarations shared by the CUDA translation units of the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <atomic>

#include "../../include/dm.h"

#define DM_MAXL 30
#define DM_MAX_LANES 4   // concurrent lanes (internal streams) of the batched form
#define DM_BATCH_MAX 8   // pairs per wave of the cross-pair batched form (one launch per step for the wave)

// Geometry of one image pair (Sec. 3.2 "Bottom level", Eq. 7, Algorithm 1).
struct DmGeom {
    int W1, H1, W2, H2;
    int L;              // top level: min{l : 4*2^l >= max(W1,H1)}, lowered to the highest level with a patch
    int P0x, P0y;       // atomic grid: centres 4k+2 <= W1-1
    int Lx, Ly;         // lattice 4Z^2 inside I: patches of levels >= 1
    int dw[DM_MAXL + 2], dh[DM_MAXL + 2];  // map domain of level l
    int key64;          // merge keys patch * |domain| + position need 64 bits (16-byte table slots)
    __host__ __device__ int npatch(int l) const { return l == 0 ? P0x * P0y : Lx * Ly; }
    __host__ __device__ int gx(int l) const { return l == 0 ? P0x : Lx; }
    __host__ __device__ long long dsize(int l) const { return (long long)dw[l] * dh[l]; }
    // row pitch (elements) of a stored pooled map on domain l: width rounded up to
    // 16, so every row of the f32 values and of the u8 argmax codes starts
    // 16-byte aligned (vector stores, 16-byte async copies, TMA tensor stores)
    __host__ __device__ int pitch(int l) const { return (dw[l] + 15) & ~15; }
    __host__ __device__ long long psize(int l) const { return (long long)pitch(l) * dh[l]; }
};

int dm_make_geom(int W1, int H1, int W2, int H2, DmGeom* g);  // 0 ok, -1 invalid, -2 unsupported

// Child i of lattice patch (ix, iy) at level l >= 1, as an index at level l-1,
// or -1 outside the grid.  o_i = (-1,-1), (-1,+1), (+1,-1), (+1,+1) as (x, y),
// child offset 2^l o_i pixels (Eq. 5).
__host__ __device__ inline int dm_child(const DmGeom& g, int l, int ix, int iy, int i) {
    int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
    if (l == 1) {
        int cx = ix + ((ox - 1) >> 1), cy = iy + ((oy - 1) >> 1);
        if (cx < 0 || cy < 0 || cx >= g.P0x || cy >= g.P0y) return -1;
        return cy * g.P0x + cx;
    }
    int s = 1 << (l - 2);
    int cx = ix + ox * s, cy = iy + oy * s;
    if (cx < 0 || cy < 0 || cx >= g.Lx || cy >= g.Ly) return -1;
    return cy * g.Lx + cx;
}

// ---------------------------------------------------------------------------
// Elementary functions with a fixed sequence of correctly rounded FP32
// operations (explicit __f*_rn intrinsics; the library is built with
// contraction off), so that any implementation of the same recipe -- the CPU
// reference in particular -- produces identical bits.
//
// dm_expf(z), z <= 0: clamp at -87; n = rint(z * log2(e)); r = z - n*ln2 with
//   ln2 split into a 16-bit head 0.693145751953125 and a tail
//   1.42860682e-06 (two fmas); e^r by the degree-7 Taylor polynomial
//   (coefficients 1/k!) in Horner form; times 2^n from the exponent field.
// dm_powf(x, lam), x in [0,1]: x = m 2^e with m in [sqrt(1/2), sqrt(2)];
//   log2 m = (2/ln2) f (1 + f^2/3 + ... + f^12/13), f = (m-1)/(m+1);
//   lam*e split exactly (product + fma residual); the exponent is reduced to
//   |g| <= 1/2 with two rint steps; 2^g by the degree-7 Taylor polynomial of
//   e^(g ln2) (coefficients ln2^k/k!); scaled by 2^n in two steps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dm_pow2i(int n) { return __int_as_float((n + 127) << 23); }

__device__ __forceinline__ float dm_expf(float z) {
    if (z < -87.0f) z = -87.0f;
    float n = rintf(__fmul_rn(z, 1.44269504f));
    float r = __fmaf_rn(n, -0.693145751953125f, z);
    r = __fmaf_rn(n, -1.42860682e-06f, r);
    float p = 1.98412698e-04f;
    p = __fmaf_rn(p, r, 1.38888889e-03f);
    p = __fmaf_rn(p, r, 8.33333333e-03f);
    p = __fmaf_rn(p, r, 4.16666667e-02f);
    p = __fmaf_rn(p, r, 1.66666667e-01f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    return __fmul_rn(p, dm_pow2i((int)n));
}

__device__ __forceinline__ float dm_powf(float x, float lam) {
    if (!(x > 0.0f)) return 0.0f;
    int eadj = 0;
    if (x < 1.17549435e-38f) { x = __fmul_rn(x, 16777216.0f); eadj = -24; }
    uint32_t b = __float_as_uint(x);
    int e = (int)((b >> 23) & 0xffu) - 127 + eadj;
    float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = __fmul_rn(m, 0.5f); e = e + 1; }
    float f = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    float f2 = __fmul_rn(f, f);
    float s = 7.69230769e-02f;
    s = __fmaf_rn(s, f2, 9.09090909e-02f);
    s = __fmaf_rn(s, f2, 1.11111111e-01f);
    s = __fmaf_rn(s, f2, 1.42857143e-01f);
    s = __fmaf_rn(s, f2, 2.00000000e-01f);
    s = __fmaf_rn(s, f2, 3.33333333e-01f);
    s = __fmaf_rn(s, f2, 1.0f);
    float l2m = __fmul_rn(__fmul_rn(2.88539008f, f), s);
    float fe = (float)e;
    float a = __fmul_rn(lam, fe);
    float aerr = __fmaf_rn(lam, fe, -a);
    float n1 = rintf(a);
    float g = __fadd_rn(__fadd_rn(__fsub_rn(a, n1), aerr), __fmul_rn(lam, l2m));
    float n2 = rintf(g);
    g = __fsub_rn(g, n2);
    float p = 1.52527338e-05f;
    p = __fmaf_rn(p, g, 1.54035304e-04f);
    p = __fmaf_rn(p, g, 1.33335581e-03f);
    p = __fmaf_rn(p, g, 9.61812911e-03f);
    p = __fmaf_rn(p, g, 5.55041087e-02f);
    p = __fmaf_rn(p, g, 2.40226507e-01f);
    p = __fmaf_rn(p, g, 6.93147181e-01f);
    p = __fmaf_rn(p, g, 1.0f);
    int nt = (int)n1 + (int)n2;
    // p in [0.70, 1.42]: for nt >= -125 the product p 2^nt is normal, so one
    // exact multiplication gives the same bits as the two-step scaling below
    if (nt >= -125) return __fmul_rn(p, dm_pow2i(nt));
    if (nt < -151) return 0.0f;
    int na = nt / 2, nb = nt - na;
    return __fmul_rn(__fmul_rn(p, dm_pow2i(na)), dm_pow2i(nb));
}

// dm_powf on two values at once: the same operations in the same order, the
// floating-point ones as packed FP32x2 instructions where both lanes do the
// same thing (each lane rounds exactly as the scalar operation would), so
// each lane's result has the bits dm_powf gives it.  No packed product feeds a
// packed addition (see the exponent reduction below).
__device__ __forceinline__ float2 dm_powf2(float2 x, float lam) {
    float2 r;
    // lanes that leave the common path (x <= 0, subnormal x, a subnormal result)
    // take the scalar recipe
    const bool fast = x.x >= 1.17549435e-38f && x.y >= 1.17549435e-38f;
    if (!fast) return make_float2(dm_powf(x.x, lam), dm_powf(x.y, lam));
    const uint32_t b0 = __float_as_uint(x.x), b1 = __float_as_uint(x.y);
    int e0 = (int)((b0 >> 23) & 0xffu) - 127, e1 = (int)((b1 >> 23) & 0xffu) - 127;
    float m0 = __uint_as_float((b0 & 0x7fffffu) | 0x3f800000u), m1 = __uint_as_float((b1 & 0x7fffffu) | 0x3f800000u);
    if (m0 > 1.41421356f) { m0 = __fmul_rn(m0, 0.5f); e0 = e0 + 1; }
    if (m1 > 1.41421356f) { m1 = __fmul_rn(m1, 0.5f); e1 = e1 + 1; }
    const float2 m = make_float2(m0, m1);
    const float2 num = __fadd2_rn(m, make_float2(-1.0f, -1.0f));
    const float2 den = __fadd2_rn(m, make_float2(1.0f, 1.0f));
    const float2 f = make_float2(__fdiv_rn(num.x, den.x), __fdiv_rn(num.y, den.y));
    const float2 f2 = __fmul2_rn(f, f);
    float2 s = make_float2(7.69230769e-02f, 7.69230769e-02f);
    s = __ffma2_rn(s, f2, make_float2(9.09090909e-02f, 9.09090909e-02f));
    s = __ffma2_rn(s, f2, make_float2(1.11111111e-01f, 1.11111111e-01f));
    s = __ffma2_rn(s, f2, make_float2(1.42857143e-01f, 1.42857143e-01f));
    s = __ffma2_rn(s, f2, make_float2(2.00000000e-01f, 2.00000000e-01f));
    s = __ffma2_rn(s, f2, make_float2(3.33333333e-01f, 3.33333333e-01f));
    s = __ffma2_rn(s, f2, make_float2(1.0f, 1.0f));
    const float2 l2m = __fmul2_rn(__fmul2_rn(make_float2(2.88539008f, 2.88539008f), f), s);
    const float2 fe = make_float2((float)e0, (float)e1);
    const float2 lam2 = make_float2(lam, lam);
    const float2 a = __fmul2_rn(lam2, fe);
    const float2 aerr = __ffma2_rn(lam2, fe, make_float2(-a.x, -a.y));
    const float2 n1 = make_float2(rintf(a.x), rintf(a.y));
    // the product lam * log2 m feeds an addition: it is formed by scalar
    // multiplications, since a packed multiplication followed by a packed
    // addition was found fused into one rounding despite contraction being off
    const float2 lg = make_float2(__fmul_rn(lam, l2m.x), __fmul_rn(lam, l2m.y));
    float2 g = __fadd2_rn(__fadd2_rn(__fadd2_rn(a, make_float2(-n1.x, -n1.y)), aerr), lg);
    const float2 n2 = make_float2(rintf(g.x), rintf(g.y));
    g = __fadd2_rn(g, make_float2(-n2.x, -n2.y));
    float2 p = make_float2(1.52527338e-05f, 1.52527338e-05f);
    p = __ffma2_rn(p, g, make_float2(1.54035304e-04f, 1.54035304e-04f));
    p = __ffma2_rn(p, g, make_float2(1.33335581e-03f, 1.33335581e-03f));
    p = __ffma2_rn(p, g, make_float2(9.61812911e-03f, 9.61812911e-03f));
    p = __ffma2_rn(p, g, make_float2(5.55041087e-02f, 5.55041087e-02f));
    p = __ffma2_rn(p, g, make_float2(2.40226507e-01f, 2.40226507e-01f));
    p = __ffma2_rn(p, g, make_float2(6.93147181e-01f, 6.93147181e-01f));
    p = __ffma2_rn(p, g, make_float2(1.0f, 1.0f));
    // n1 + n2 is a sum of two small integers, exact in FP32: one conversion per lane
    const float2 ntf = __fadd2_rn(n1, n2);
    const int nt0 = (int)ntf.x, nt1 = (int)ntf.y;
    if (nt0 >= -125 && nt1 >= -125) return __fmul2_rn(p, make_float2(dm_pow2i(nt0), dm_pow2i(nt1)));
    // a result below the normal range: the scalar two-step scaling per lane
    r.x = dm_powf(x.x, lam);
    r.y = dm_powf(x.y, lam);
    return r;
}

// ---------------------------------------------------------------------------
// Workspace layouts (all offsets 256-byte aligned).
// ---------------------------------------------------------------------------
static inline size_t dm_align(size_t v) { return (v + 255) & ~(size_t)255; }

// Header at offset 0 of backtracking and dm_match workspaces.
struct DmWsHeader {
    int status;                   // DM_DEV_* bits of the backtracking step
    int pyr_status;               // nonzero: a bounded wait of a pyramid kernel gave up
    int pad0[14];
    unsigned int count[DM_MAXL + 2];   // merged tuples per level (level 0: arrivals)
    unsigned int cap[DM_MAXL + 2];     // active merge-table capacity per level
    unsigned int entries[DM_MAXL + 2]; // DM*: local-maximum entry points per level
};

struct DmPyrLayout {
    size_t header;                // DmWsHeader (pyr_status used)
    size_t valid[DM_MAXL + 1];    // u8 [npatch(l)]
    size_t pooled[DM_MAXL];       // f32 [npatch(l)][dh[l+1]][pitch(l+1)]
    size_t amax[DM_MAXL];         // u8 same shape
    size_t top;                   // f32 [npatch(L)][dh[L]][dw[L]]
    size_t a16;                   // packed patch operand tiles of the tensor-core forms (BF16, E4M3 + scales)
    size_t bytes;
};

struct DmBtLayout {
    size_t header;                // DmWsHeader
    size_t table[DM_MAXL + 1];    // u64 merge tables, levels 1..L-1
    size_t cap[DM_MAXL + 1];      // max slots per level
    size_t bestP, bestQ;          // u64 keys
    size_t elist[DM_MAXL + 1];    // DM*: entry points found per level, u64 (key << 32 | score)
    size_t elcap[DM_MAXL + 1];    // DM*: their capacity (entries)
    size_t bytes;
};

// Workspace of the differentiable form (gradient of the top-maxima loss).
#define DM_GRAD_COUNTS (2 * DM_MAXL + 4)
struct DmGradLayout {
    size_t parts;                 // f32 [npatch(L)] per-patch maxima
    size_t dA[DM_MAXL + 1];       // f32 [npatch(l)][dh[l]][dw[l]], l = 1..L
    size_t dP[DM_MAXL];           // f32 pooled layout, l = 0..L-1
    size_t Am, Bm;                // f32 [n0][144] patch vectors, [W2*H2][144] image-2 im2col
    size_t G1, Gim;               // f32 [n0][144], [W2*H2][144] level-0 products
    size_t box;                   // int4 [n0] bounding box of each patch's level-0 argmax positions
    size_t box0;                  // int4 [n0] box of the nonzeros of dP_0 per patch (x0, y0, -x1, -y1)
    size_t frontE, frontF;        // int2 [cap] frontiers (patch, position) of the nonzeros of dA_l / dP_l
    size_t counts;                // u32 [DM_GRAD_COUNTS] frontier sizes per level, then an overflow flag
    unsigned int cap;             // entries per frontier buffer (bounds every frontier: no overflow)
    bool cap_ok;                  // false: a frontier could exceed 2^32 entries (refused)
    size_t bytes;
};

void dm_pyr_layout(const DmGeom& g, int precision, DmPyrLayout* o);
void dm_grad_layout(const DmGeom& g, DmGradLayout* o);
// star: the DM* variant's tables (levels 1..L, room for the entry points too)
void dm_bt_layout(const DmGeom& g, DmBtLayout* o, bool star = false);
size_t dm_desc_tmp_bytes(int W, int H);

// Suspend-time hint of the kernels' mbarrier waits: a waiting thread sleeps
// until the phase completes (or this many ns pass) instead of spinning and
// taking issue slots from the warps that do the work.
constexpr unsigned WAIT_HINT_NS = 1000000u;

// Launch shapes the autotuner chooses among (every choice computes identical
// results): M-tiles of 128 patches per work unit of the tensor-core level-0
// kernel, pooled rows per CTA tile of the level kernel (8 or 16), CTAs per SM
// of the backtracking expansion kernels, child-window columns in the level
// kernel's ring (3 or 2: prefetch depth against shared memory per CTA).
struct DmTune {
    int m_chunk;
    int level_th;
    int bt_mult;
    int level_ring;
};
// Defaults until tuned: the level-0 work unit holds all M-tiles of the pair
// (the N-tiles are the units; measured at 1024x436 the most robust choice for
// BF16) or, for the FP8 form, half of them (its best measured split); tile
// rows 8 (on 4 warps; 1024x436: 7.79 ms against 8.31 for 16 rows on 8 warps,
// 8.71 for 4 rows on 2), 8 CTAs per SM for the backtracking, a ring of 2.
inline DmTune dm_tune_default(const DmGeom& g, int precision) {
    const int n_mtiles = (g.npatch(0) + 127) / 128;
    return DmTune{precision == DM_FP8_E4M3 ? (n_mtiles + 1) / 2 : n_mtiles, 8, 8, 2};
}

// Pyramid handle (host side).
struct dm_pyramid {
    DmGeom g;
    int precision;
    int compensated;              // child sums of Eq. 12: TwoSum-compensated (1) or plain (0)
    DmTune tune;                  // launch shapes for this pair's size
    const unsigned char* valid[DM_MAXL + 1];
    const float* pooled[DM_MAXL];
    const unsigned char* amax[DM_MAXL];
    const float* top;
    // approximate form (Sec. 4.1): level 0 holds one map per prototype and
    // atomic patch c reads map proto_of[c] (caller-owned device array);
    // exact form: proto_of = nullptr, n0_maps = npatch(0)
    const int* proto_of;
    int n0_maps;
    // fault injection (dm_inject_fault): > 0, every CTA of the level kernel
    // first waits this many cycles on a barrier nothing completes, so its
    // bounded wait runs out and the pyramid status reports it; 0 otherwise
    long long inject_wait;
};

// ---------------------------------------------------------------------------
// Average of a lattice patch's children at one position (Eq. 12, boundary
// rule): C_l(p, q) before rectification = (1/n) sum over the n existing
// children c_i of P_{l-1}(c_i, q + o_i), 0 outside the domain.  Shared by the
// top level and the local-maximum search of DM*, so that both produce the
// averages of the level pass bit for bit.
// ---------------------------------------------------------------------------
struct Kids {
    const float* base[4];
    int n;
};

// a - b for two lanes at once, each lane rounded as the scalar subtraction
// (the packed add has no negated operand, so a - b written as a + (-b) would
// need the negations as separate instructions)
__device__ __forceinline__ float2 dm_fsub2(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    memcpy(&ra, &a, 8);
    memcpy(&rb, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    memcpy(&d, &rd, 8);
    return d;
}

// One packed step of Knuth's TwoSum (s, x) -> (s + x, its rounding error),
// two lanes at once; every operation rounded as the scalar one.
__device__ __forceinline__ void dm_two_sum2(float2& s, float2 x, float2& err) {
    const float2 t = __fadd2_rn(s, x);
    const float2 bp = dm_fsub2(t, s);
    const float2 e1 = dm_fsub2(s, dm_fsub2(t, bp));
    const float2 e2 = dm_fsub2(x, bp);
    err = __fadd2_rn(e1, e2);
    s = t;
}

// One step of the compensated child sum (Knuth's TwoSum gives the same bits
// for any operands): for non-negative operands, which every map value is,
// Dekker's Fast2Sum on (max, min) is exact, since the first operand is the
// larger, with one operation fewer.
__device__ __forceinline__ void fast_two_sum_add(float& s, float& comp, float v) {
    const float hi = fmaxf(s, v), lo = fminf(s, v);
    const float t = __fadd_rn(hi, lo);
    const float err = __fsub_rn(lo, __fsub_rn(t, hi));
    s = t;
    comp = __fadd_rn(comp, err);
}

// Child sum step: compensated or plain.  The first existing child starts the
// sum (0 + v = v exactly, the same as starting from zero).
template <bool COMP>
__device__ __forceinline__ void child_add(float& s, float& comp, float v) {
    if (COMP) fast_two_sum_add(s, comp, v);
    else s = __fadd_rn(s, v);
}

template <bool COMP>
__device__ __forceinline__ float child_mean(const Kids& k, int qx, int qy, int mw, int mh, int pitch) {
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (k.base[i] == nullptr) continue;
        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        int rx = qx + ox, ry = qy + oy;
        float v = 0.0f;
        if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) v = __ldg(k.base[i] + (long long)ry * pitch + rx);
        child_add<COMP>(s, comp, v);
    }
    return __fdiv_rn(__fadd_rn(s, comp), (float)k.n);
}


// (proto_of: the map of atomic child c is map proto_of[c], clamped to
// [0, n_maps) -- approximate form, l = 1)
__device__ __forceinline__ bool load_kids(const DmGeom& g, int l, int p, const unsigned char* __restrict__ vprev,
                                          const float* __restrict__ prev, Kids& k, const int* __restrict__ proto_of,
                                          int n_maps) {
    int ix = p % g.Lx, iy = p / g.Lx;
    long long cs = g.psize(l);     // child pooled map size (domain of level l, padded rows)
    k.n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int c = dm_child(g, l, ix, iy, i);
        if (c >= 0 && vprev[c]) {
            k.base[i] = prev + (long long)(proto_of ? min(max(proto_of[c], 0), n_maps - 1) : c) * cs;
            k.n++;
        } else {
            k.base[i] = nullptr;
        }
    }
    return k.n > 0;
}

// ---------------------------------------------------------------------------
// Scale and rotation invariant form (Sec. 4.2, Algorithm 2).
//
// A warped canvas Wr x Hr holds an image W x H downsized by sigma and rotated
// by -theta.  Canvas pixel (u, v) samples the image at
//   (x, y) = image centre + sigma * R_theta * ((u, v) - canvas centre);
// the same map takes a canvas position back to the image when the atomic
// correspondences are rectified.  The order of the rounded FP32 operations is
// part of the definition: the warp and the rectification use this one
// function.
struct DmXform {
    float cu, cv;      // canvas centre ((Wr - 1) / 2, (Hr - 1) / 2)
    float cx, cy;      // image centre ((W - 1) / 2, (H - 1) / 2)
    float sg, c, s;    // sigma, cos theta, sin theta
};

__device__ __forceinline__ void dm_to_source(const DmXform& t, float u, float v, float& x, float& y) {
    const float du = __fsub_rn(u, t.cu), dv = __fsub_rn(v, t.cv);
    const float rx = __fsub_rn(__fmul_rn(t.c, du), __fmul_rn(t.s, dv));
    const float ry = __fadd_rn(__fmul_rn(t.s, du), __fmul_rn(t.c, dv));
    x = __fadd_rn(t.cx, __fmul_rn(t.sg, rx));
    y = __fadd_rn(t.cy, __fmul_rn(t.sg, ry));
}

// Rectification of one transform's atomic correspondences to the input pair:
// a correspondence (patch c of the warped image 1, canvas pixel t of the warped
// image 2, score s) becomes (the atomic patch of I holding sigma1 * centre(c),
// the pixel of I' nearest sigma2 R_theta t) and is reduced into the input
// pair's BestAt / BestAt' arrays.
struct DmRect {
    DmXform t1, t2;               // warped image 1 (theta = 0) and warped image 2
    int W1, H1, W2, H2;           // input sizes
    int P0x, P0y;                 // atomic lattice of the input image 1
    unsigned long long* bestP;    // BestAt of the input pair  [P0x * P0y]
    unsigned long long* bestQ;    // BestAt' of the input pair [ceil(W2/4) * ceil(H2/4)]
};

// Transform i (0..71) of Algorithm 2's list: sigma = -2 + 0.5 (i / 8) (outer),
// theta = (i % 8) pi/4 (inner); sigma1 = max(1, 2^sigma) downsizes image 1,
// sigma2 = max(1, 2^-sigma) image 2; (w1, h1), (w2, h2) are the canvas sizes.
struct DmInvTransform {
    double s1, s2;
    int k;
    int w1, h1, w2, h2;
};
constexpr int DM_INV_TRANSFORMS = 72;
void dm_invariant_transform(int i, int W1, int H1, int W2, int H2, DmInvTransform* t);
DmXform dm_make_xform(int W, int H, int Wr, int Hr, double sigma, int k);
cudaError_t dm_launch_warp(const float* img, int W, int H, float* out, int Wr, int Hr, const DmXform& t,
                           cudaStream_t st);
// dst->status |= src->status, dst->pyr_status |= src->pyr_status and the
// per-level counts added (saturating), all atomically: one transform's outcome
// folded into the invariant call's header (transforms may run concurrently).
cudaError_t dm_launch_inv_fold(DmWsHeader* dst, const DmWsHeader* src, cudaStream_t st);

// Smoothing taps passed by value to kernels.
struct DmTaps {
    int R;
    float w[65];
};

struct DmDescParams {
    DmTaps t1, t2, t3;
    float scale, slope, mu;
};

// DeepFlow (Sec. 4.3), see k_deepflow.cu.
#define DM_DF_MAXLEVELS 256
struct DmFlowPlan {
    int nl;                                   // levels (k_max + 1), finest first
    int ws[DM_DF_MAXLEVELS], hs[DM_DF_MAXLEVELS];
    float beta_k[DM_DF_MAXLEVELS], sk[DM_DF_MAXLEVELS];   // matching weight and eta^k per level
    float eta, inv_eta, scale, kappa, gamma, delta, zeta2, eps2, omega, one_m_omega, sigma_m, two_sigma_m, norm;
    int n_fixed, n_sor, capacity;
    size_t P1[DM_DF_MAXLEVELS], P2[DM_DF_MAXLEVELS];      // workspace offsets
    size_t tmp, fa_u, fa_v, fb_u, fb_v, du, dv, du2, dv2, alpha, I2w, Im, Ix, Iy, ps, mc, mu, mv, D, A, owner, phi;
    size_t bytes;
};
void dm_flow_plan(int W, int H, int capacity, const dm_flow_params& p, DmFlowPlan* q);
cudaError_t dm_launch_smooth1(const float* img, int W, int H, float scale, const DmTaps& t, float* out, float* tmp,
                              cudaStream_t st);
cudaError_t dm_launch_deepflow(const DmFlowPlan& q, const DmTaps& taps, const float* img1, const float* img2,
                               const dm_match_t* m, const int* d_count, float* out_u, float* out_v, char* ws,
                               cudaStream_t st);

// Record an error message on a context and return `s`; device of a context.
dm_status dm_set_error(dm_ctx* ctx, dm_status s, const char* msg);
int dm_ctx_device(const dm_ctx* ctx);

// Number of kernels the library has launched in this process (host counter,
// advanced by each launcher).
void dm_count_launches(long long n);
long long dm_launches();

// Opt `kernel` into `bytes` of dynamic shared memory on the current device,
// once per device (`done` holds one bit per device below 64; other devices
// set the attribute on every call).  Thread-safe.
inline cudaError_t dm_smem_opt_in(const void* kernel, int bytes, std::atomic<unsigned long long>& done) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
    return e;
}

// Tiled tensor map (cuTensorMapEncodeTiled, reached through the runtime's
// driver entry point): no interleave, the given shared-memory swizzle (none by
// default), zero fill outside the extent, element strides 1.  False if the
// entry point is unavailable or the map is rejected (base not 16-byte aligned,
// stride not a multiple of 16 B, box row wider than the swizzle span, ...).
bool dm_encode_tiled(CUtensorMap* m, CUtensorMapDataType dt, int rank, void* base, const cuuint64_t* dims,
                     const cuuint64_t* strides_bytes, const cuuint32_t* box,
                     CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE);

// Kernel launchers (return cudaGetLastError()).
cudaError_t dm_launch_descriptors(const DmDescParams& prm, const float* img, int W, int H, float* desc,
                                  float* tmpA, float* tmpB, cudaStream_t st);
// The same for n <= 2 DM_BATCH_MAX images: one launch per pass for all of them.
cudaError_t dm_launch_descriptors_batch(const DmDescParams& prm, int n, const float* const* imgs, const int* Ws,
                                        const int* Hs, float* const* descs, float* const* tmpAs, float* const* tmpBs,
                                        cudaStream_t st);
// Level-0 launchers.  The rows of the correlation are image 1's atomic
// patches taken from d1, or, when amat is given, the n_rows vectors
// amat[n_rows][144] (k = (dy*4 + dx)*9 + c; the prototypes of the approximate
// form), whose maps then fill rows 0 .. n_rows-1 of the level-0 arrays.
cudaError_t dm_launch_corr0_f32(const DmGeom& g, const float* d1, const float* d2, float lam, float* pooled0,
                                unsigned char* amax0, cudaStream_t st, const float* amat = nullptr, int n_rows = -1);
// tcgen05 level-0 correlation, precision DM_BF16 or DM_FP8_E4M3; abuf holds
// dm_corr0_tc_a_bytes(g, precision) bytes of packed operands.
cudaError_t dm_launch_corr0_tc(const DmGeom& g, int precision, const float* d1, const float* d2, float lam, void* abuf,
                               void* status, float* pooled0, unsigned char* amax0, int m_chunk, cudaStream_t st,
                               const float* amat = nullptr, int n_rows = -1);
// Level 0 of the n <= DM_BATCH_MAX pairs of a wave (exact form): their operand
// packing, then one persistent launch that drains the work units of all pairs.
cudaError_t dm_launch_corr0_tc_batch(int n, const DmGeom* gs, int precision, const float* const* d1s,
                                     const float* const* d2s, float lam, void* const* abufs, void* const* statuses,
                                     float* const* pooled0s, unsigned char* const* amax0s, const int* m_chunks,
                                     cudaStream_t st);
// Spherical k-means of image 1's atomic patches (Sec. 4.1), see k_approx.cu.
size_t dm_kmeans_ws_bytes(const DmGeom& g, int D);
size_t dm_kmeans_init_offset(const DmGeom& g, int D);
cudaError_t dm_launch_kmeans(const DmGeom& g, const float* d1, int D, int iters, const int* init, float* protos,
                             int* assign, char* ws, cudaStream_t st);
size_t dm_corr0_tc_a_bytes(const DmGeom& g, int precision);
cudaError_t dm_launch_levels(const DmGeom& g, const dm_pyramid& p, float lam, int* status, cudaStream_t st);
// The same for the n <= DM_BATCH_MAX pyramids of a wave (same precision and
// child-sum mode, level 0 computed): one launch per kernel and level for all.
cudaError_t dm_launch_levels_batch(const dm_pyramid* const* pys, int n, float lam, int* const* status, cudaStream_t st);
cudaError_t dm_launch_loss_grad(const DmGeom& g, const dm_pyramid& py, const float* d1, const float* d2, float lam,
                                const DmGradLayout& gl, char* ws, float* d_loss, float* g1, float* g2, cudaStream_t st);
// With rect != nullptr the atomic correspondences are rectified into
// rect->bestP / rect->bestQ (which the caller clears once) and no reciprocal
// step runs: out, capacity and d_count are unused.
cudaError_t dm_launch_backtrack(const DmGeom& g, const dm_pyramid& p, const DmBtLayout& bl, char* ws,
                                dm_match_t* out, int capacity, int* d_count, cudaStream_t st,
                                const DmRect* rect = nullptr);
// The same for the n <= DM_BATCH_MAX pairs of a wave (pyramids computed), each
// with its own workspace wss[j] (layout *bls[j]) and output: one launch per
// step of the descent for all of them, then one reciprocal launch.
cudaError_t dm_launch_backtrack_batch(const dm_pyramid* const* pys, const DmBtLayout* const* bls, char* const* wss,
                                      dm_match_t* const* outs, const int* caps, int* const* counts, int n, cudaStream_t st);
// DM* (Sec. 5.3): entry points at the local maxima of every level's maps,
// start + end scoring; bl from dm_bt_layout(g, &bl, true).
cudaError_t dm_launch_backtrack_star(const DmGeom& g, const dm_pyramid& p, const DmBtLayout& bl, char* ws, float lam,
                                     dm_match_t* out, int capacity, int* d_count, cudaStream_t st);
// Reciprocal verification (Eq. 16) of BestAt / BestAt' arrays of geometry g.
cudaError_t dm_launch_reciprocal(const DmGeom& g, unsigned long long* bestP, unsigned long long* bestQ, DmWsHeader* hdr,
                                 dm_match_t* out, int capacity, int* d_count, cudaStream_t st);
