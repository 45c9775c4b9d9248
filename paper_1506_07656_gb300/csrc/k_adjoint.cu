// Differentiable form: loss = sum over existing top patches p of
// max_q C_L(p, q) (first maximum), and its gradient with respect to both
// descriptor fields (the paper has no loss; this is the adjoint of
// Algorithm 1).  The backward runs through
//   the rectification  C = A^lambda                  (Eq. 11),
//   the shifted average A_l = mean_i P_{l-1}(c_i, q+o_i)   (Eq. 12),
//   the max-pooling with its saved argmax            (Eq. 8-9),
//   the level-0 correlation C0 = (1/16) a_p . b_t    (Eq. 3-4).
// Everything is a gather with a fixed summation order, so the gradient is
// deterministic.  Per level two dense arrays are used: dA_l on the map
// domain of level l (unrectified averages) and dP_l in the pooled layout.
// Level 0 is recomputed rather than stored: the unrectified C0 at an argmax
// position is one 144-term dot product.  Of the two level-0 products
//   G1[p][k] = (1/16) sum_t dC0(p,t) b_t[k],   Gim[t][k] = (1/16) sum_p dC0(p,t) a_p[k]
// both are gathers over the nonzeros of dC0 (at most one per pooled output):
// G1 one warp per patch, which also leaves each pooled output's coefficient
// in place of dP0 and the bounding box of the patch's argmax positions; Gim
// one warp per row segment of 30 positions of I', which visits, in patch
// order, the patches whose box meets the segment.  Then G1 is scattered onto
// the atomic windows of I and Gim gathered (col2im) onto the pixels of I'.
#include "dm_internal.cuh"

namespace {

// Unrectified average of lattice patch p at level l >= 1, position (qx, qy),
// exactly as the forward computes it (child order, TwoSum-compensated when
// `comp`); *n_out = number of existing children.
__device__ float level_average(const DmGeom& g, int l, int p, int qx, int qy, const unsigned char* vprev,
                               const float* prev, bool comp, int* n_out) {
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);
    float s = 0.0f, c = 0.0f;
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int ch = dm_child(g, l, p % g.Lx, p / g.Lx, i);
        if (ch < 0 || !vprev[ch]) continue;
        n++;
        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        int rx = qx + ox, ry = qy + oy;
        float v = 0.0f;
        if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) v = prev[(long long)ch * g.psize(l) + (long long)ry * pitch + rx];
        const float t = __fadd_rn(s, v);
        if (comp) {
            const float bp = __fsub_rn(t, s);
            c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp)));
        }
        s = t;
    }
    *n_out = n;
    if (n == 0) return 0.0f;
    return __fdiv_rn(__fadd_rn(s, c), (float)n);
}

__device__ __forceinline__ float dpow(float x, float lam) {   // d(x^lam)/dx for x in [0, 1]
    return x > 0.0f ? __fmul_rn(lam, dm_powf(x, lam - 1.0f)) : 0.0f;
}

// Top level: per existing patch, the first maximum of C_L, its value, and
// dA_L = d(A^lam)/dA at that position (zero elsewhere).
__global__ void k_adj_top(DmGeom g, const unsigned char* __restrict__ vL, const unsigned char* __restrict__ vprev,
                          const float* __restrict__ top, const float* __restrict__ prev, float lam, int comp,
                          float* __restrict__ dA, float* __restrict__ parts, int4* __restrict__ boxL) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int L = g.L;
    if (p >= g.npatch(L)) return;
    const int nq = g.dw[L] * g.dh[L];
    float* d = dA + (long long)p * nq;
    for (int q = 0; q < nq; q++) d[q] = 0.0f;
    if (!vL[p]) { parts[p] = 0.0f; boxL[p] = make_int4(0, 0, -1, -1); return; }
    const float* t = top + (long long)p * nq;
    float best = -INFINITY;
    int qb = 0;
    for (int q = 0; q < nq; q++)
        if (t[q] > best) { best = t[q]; qb = q; }
    parts[p] = best;
    int n;
    const float a = level_average(g, L, p, qb % g.dw[L], qb / g.dw[L], vprev, prev, comp != 0, &n);
    d[qb] = dpow(a, lam);
    boxL[p] = make_int4(qb % g.dw[L], qb / g.dw[L], qb % g.dw[L], qb / g.dw[L]);
}

// Deterministic sum of the per-patch maxima (one block).
__global__ void k_adj_loss(const float* __restrict__ parts, int n, float* __restrict__ loss) {
    __shared__ double acc[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)parts[i];
    acc[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) acc[threadIdx.x] += acc[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)acc[0];
}

// Parent i (0..3) of child c at level l (c at level l - 1), or -1 where the
// child is not valid, the parent lies outside the lattice or is not valid;
// *n = the parent's number of valid children (the divisor of its average).
__device__ int adj_parent(const DmGeom& g, int l, int c, int i, const unsigned char* vcur,
                          const unsigned char* vprev, int* n) {
    *n = 0;
    if (!vprev[c]) return -1;
    const int cx = l == 1 ? c % g.P0x : c % g.Lx, cy = l == 1 ? c / g.P0x : c / g.Lx;
    const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
    int ix, iy;
    if (l == 1) { ix = cx + (1 - ox) / 2; iy = cy + (1 - oy) / 2; }
    else { const int s = 1 << (l - 2); ix = cx - ox * s; iy = cy - oy * s; }
    if (ix < 0 || iy < 0 || ix >= g.Lx || iy >= g.Ly) return -1;
    const int p = iy * g.Lx + ix;
    if (!vcur[p]) return -1;
    for (int j = 0; j < 4; j++) {
        const int cj = dm_child(g, l, ix, iy, j);
        if (cj >= 0 && vprev[cj]) (*n)++;
    }
    return p;
}

__device__ __forceinline__ bool in_box(const int4& b, int x, int y) {
    return x >= b.x && x <= b.z && y >= b.y && y <= b.w;
}

// Support boxes of the gradient, one step down from level l: for child c,
// par[c] / nch[c] receive its four parents (adj_parent) and their divisors;
// boxP[c] bounds the pooled positions r where dP_{l-1}(c, r) can be nonzero
// (the parents' boxes of dA_l shifted by their offsets o_i), and, where
// m = l - 1 >= 1, boxAm[c] bounds the positions t = 2r + (-1..1) of domain m
// where dA_m(c, t) can be nonzero.  Supersets: outside them every term of the
// gathers below is an exact zero, so skipping them leaves every sum unchanged.
__global__ void k_adj_box(DmGeom g, int l, const unsigned char* __restrict__ vcur, const unsigned char* __restrict__ vprev,
                          const int4* __restrict__ boxA, int4* __restrict__ boxP, int4* __restrict__ boxAm,
                          int4* __restrict__ par, int4* __restrict__ nch) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= g.npatch(l - 1)) return;
    int x0 = INT_MAX, y0 = INT_MAX, x1 = -1, y1 = -1;
    int pi[4], ni[4];
    for (int i = 0; i < 4; i++) pi[i] = adj_parent(g, l, c, i, vcur, vprev, &ni[i]);
    par[c] = make_int4(pi[0], pi[1], pi[2], pi[3]);
    nch[c] = make_int4(ni[0], ni[1], ni[2], ni[3]);
    for (int i = 0; i < 4; i++) {
        const int p = pi[i];
        if (p < 0) continue;
        const int4 b = boxA[p];
        if (b.x > b.z || b.y > b.w) continue;
        const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        x0 = min(x0, b.x + ox); x1 = max(x1, b.z + ox);
        y0 = min(y0, b.y + oy); y1 = max(y1, b.w + oy);
    }
    x0 = max(x0, 0); y0 = max(y0, 0);
    x1 = min(x1, g.dw[l] - 1); y1 = min(y1, g.dh[l] - 1);
    boxP[c] = make_int4(x0, y0, x1, y1);
    if (boxAm) {
        const int m = l - 1;
        if (x0 > x1 || y0 > y1) boxAm[c] = make_int4(0, 0, -1, -1);
        else boxAm[c] = make_int4(max(2 * x0 - 1, 0), max(2 * y0 - 1, 0), min(2 * x1 + 1, g.dw[m] - 1),
                                  min(2 * y1 + 1, g.dh[m] - 1));
    }
}

constexpr int ADJ_PPT = 8;   // positions per thread of the per-level passes

// dP_{l-1}(c, r) = sum over the parents p_i = c - 2^l o_i of c (i = 0..3, in
// order) of dA_l(p_i, r - o_i) / n(p_i).  Grid: (runs of 128 * ADJ_PPT
// positions of domain l, child); par / nch from k_adj_box.  Positions outside
// the child's support box, and parent positions outside the parent's,
// contribute exact zeros and are not read.
__global__ void __launch_bounds__(128) k_adj_pooled(DmGeom g, int l, const float* __restrict__ dA, float* __restrict__ dP,
                                                    const int4* __restrict__ boxA, const int4* __restrict__ boxP,
                                                    const int4* __restrict__ par, const int4* __restrict__ nch) {
    const int c = blockIdx.y;
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);
    const int n = mw * mh;
    float* out = dP + (long long)c * g.psize(l);
    const int4 bp = boxP[c];
    const int4 pp = par[c], nn = nch[c];
    const int pa[4] = {pp.x, pp.y, pp.z, pp.w};
    const int na[4] = {nn.x, nn.y, nn.z, nn.w};
    const int r0 = blockIdx.x * (128 * ADJ_PPT) + threadIdx.x;
#pragma unroll 2
    for (int j = 0; j < ADJ_PPT; j++) {
        const int r = r0 + 128 * j;
        if (r >= n) break;
        const int rx = r % mw, ry = r / mw;
        float sum = 0.0f;
        if (in_box(bp, rx, ry)) {
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int p = pa[i];
                if (p < 0) continue;
                const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
                const int qx = rx - ox, qy = ry - oy;
                if (qx < 0 || qy < 0 || qx >= mw || qy >= mh) continue;
                if (!in_box(boxA[p], qx, qy)) continue;
                const float d = dA[((long long)p * mh + qy) * mw + qx];
                if (d != 0.0f) sum = __fadd_rn(sum, __fdiv_rn(d, (float)na[i]));
            }
        }
        out[(long long)ry * pitch + rx] = sum;
    }
}

// dA_{m}(c, t) for m = l-1 >= 1: sum over the pooled positions r whose argmax
// is t (r = floor/ceil(t/2) per axis, ascending) of dP_m(c, r) * lam A^(lam-1),
// A the unrectified average at t.  Grid: (positions of domain m, patch).
__global__ void __launch_bounds__(128) k_adj_unpool(DmGeom g, int m, const unsigned char* __restrict__ vm,
                                                    const unsigned char* __restrict__ vprev,
                                                    const float* __restrict__ prev, const float* __restrict__ dP,
                                                    const unsigned char* __restrict__ amax, float lam, int comp,
                                                    float* __restrict__ dA, const int4* __restrict__ boxAm) {
    const int c = blockIdx.y;
    const int tw = g.dw[m], th = g.dh[m];
    const int pw = g.dw[m + 1], ph = g.dh[m + 1], pitch = g.pitch(m + 1);
    const int4 bb = boxAm[c];
    const bool live = vm[c] != 0;
    const int t0 = blockIdx.x * (128 * ADJ_PPT) + threadIdx.x;
    for (int j = 0; j < ADJ_PPT; j++) {
        const int t = t0 + 128 * j;
        if (t >= tw * th) break;
        const int tx = t % tw, ty = t / tw;
        float sum = 0.0f;
        if (live && in_box(bb, tx, ty)) {
            float dsum = 0.0f;
            for (int ry = ty >> 1; ry <= (ty + 1) >> 1; ry++) {
                if (ry >= ph) continue;
                for (int rx = tx >> 1; rx <= (tx + 1) >> 1; rx++) {
                    if (rx >= pw) continue;
                    const long long o = (long long)c * g.psize(m + 1) + (long long)ry * pitch + rx;
                    const int code = amax[o];
                    if (2 * rx + code % 3 - 1 != tx || 2 * ry + code / 3 - 1 != ty) continue;
                    dsum = __fadd_rn(dsum, dP[o]);
                }
            }
            if (dsum != 0.0f) {
                int n;
                const float a = level_average(g, m, c, tx, ty, vprev, prev, comp != 0, &n);
                sum = __fmul_rn(dsum, dpow(a, lam));
            }
        }
        dA[((long long)c * th + ty) * tw + tx] = sum;
    }
}

// Patch vectors (A, [n0][144]) and the image-2 im2col (B, [W2*H2][144]) in FP32,
// k = (dy*4 + dx)*9 + c; zero outside the images.
__global__ void k_adj_im2col(DmGeom g, const float* __restrict__ d1, const float* __restrict__ d2,
                             float* __restrict__ Am, float* __restrict__ Bm) {
    const long long n0 = g.npatch(0), T = (long long)g.W2 * g.H2;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (n0 + T) * 144) return;
    const int k = (int)(idx % 144);
    const long long row = idx / 144;
    const int dy = k / 36, dx = (k / 9) % 4, ch = k % 9;
    if (row < n0) {
        const int p = (int)row;
        const int x = 4 * (p % g.P0x) + dx, y = 4 * (p / g.P0x) + dy;
        Am[row * 144 + k] = (x < g.W1 && y < g.H1) ? d1[((long long)y * g.W1 + x) * 9 + ch] : 0.0f;
    } else {
        const long long t = row - n0;
        const int tx = (int)(t % g.W2), ty = (int)(t / g.W2);
        const int x = tx - 2 + dx, y = ty - 2 + dy;
        Bm[t * 144 + k] = (x >= 0 && y >= 0 && x < g.W2 && y < g.H2) ? d2[((long long)y * g.W2 + x) * 9 + ch] : 0.0f;
    }
}

// G1[p][k] = (1/16) sum over the pooled positions r of patch p (row-major order)
// with dP0(p, r) != 0 of dP0(p, r) * lam C0(p, t_r)^(lam-1) * b_{t_r}[k], t_r the
// argmax position of r -- the level-0 product dC0 * B restricted to its
// nonzeros (at most one per pooled output; dC0 is zero elsewhere).  One warp
// per patch: lanes scan 32 pooled positions at a time, the warp takes their
// nonzeros in order; lane j holds k = j + 32 i (i < 5) of the accumulator and
// of the dot product C0 = (1/16) a_p . b_t (lane partials, then a fixed
// butterfly sum).  Deterministic: a fixed order throughout.
// Only the support box of dP0 (k_adj_box) is scanned.
// Each nonzero dP0(p, r) is replaced by its coefficient c = dP0(p, r) *
// lam C0(p, t_r)^(lam-1) (0 where the argmax lies outside I'), and box[p]
// receives the bounding box (x0, y0, x1, y1) of the patch's positions t_r
// (empty: x0 > x1), for the transposed product.
__global__ void __launch_bounds__(256) k_adj_g1_sparse(DmGeom g, float* __restrict__ dP0,
                                                      const unsigned char* __restrict__ amax0,
                                                      const float* __restrict__ Am, const float* __restrict__ Bm,
                                                      float lam, float* __restrict__ G1, int4* __restrict__ box,
                                                      const int4* __restrict__ boxP0) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= g.npatch(0)) return;
    const int pitch = g.pitch(1), W2 = g.W2;
    // the pooled positions outside the support box of dP0 hold exact zeros:
    // the scan covers the box only, row-major as over the whole map
    const int4 sb = boxP0[p];
    const int bw = sb.z >= sb.x ? sb.z - sb.x + 1 : 0;
    const int bh = sb.w >= sb.y ? sb.w - sb.y + 1 : 0;
    float* dp = dP0 + (long long)p * g.psize(1);
    const unsigned char* am = amax0 + (long long)p * g.psize(1);
    float a[5], acc[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int k = lane + 32 * i;
        a[i] = k < 144 ? __ldg(Am + (long long)p * 144 + k) : 0.0f;
        acc[i] = 0.0f;
    }
    int bx0 = INT_MAX, by0 = INT_MAX, bx1 = -1, by1 = -1;
    const int n = bw * bh;
    for (int r0 = 0; r0 < n; r0 += 32) {
        const int r = r0 + lane;
        float d = 0.0f;
        int t = 0;
        long long o = 0;
        bool had = false;
        if (r < n) {
            const int rx = sb.x + r % bw, ry = sb.y + r / bw;
            o = (long long)ry * pitch + rx;
            d = dp[o];
            had = d != 0.0f;
            if (had) {
                const int code = am[o];
                const int tx = 2 * rx + code % 3 - 1, ty = 2 * ry + code / 3 - 1;
                // (the forward's pooling only ever points inside I')
                if (code <= 8 && tx >= 0 && ty >= 0 && tx < W2 && ty < g.H2) {
                    t = ty * W2 + tx;
                    bx0 = min(bx0, tx); bx1 = max(bx1, tx);
                    by0 = min(by0, ty); by1 = max(by1, ty);
                } else {
                    d = 0.0f;
                }
            }
        }
        float myc = 0.0f;
        unsigned int nz = __ballot_sync(0xffffffffu, d != 0.0f);
        while (nz) {
            const int src = __ffs(nz) - 1;
            nz &= nz - 1;
            const float dv = __shfl_sync(0xffffffffu, d, src);
            const int tv = __shfl_sync(0xffffffffu, t, src);
            const float* b = Bm + (long long)tv * 144;
            float bk[5], part = 0.0f;
#pragma unroll
            for (int i = 0; i < 5; i++) {
                const int k = lane + 32 * i;
                bk[i] = k < 144 ? __ldg(b + k) : 0.0f;
                part = __fmaf_rn(a[i], bk[i], part);
            }
#pragma unroll
            for (int o2 = 16; o2 > 0; o2 >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o2));
            const float c = __fmul_rn(dv, dpow(__fmul_rn(part, 0.0625f), lam));   // this r's share of dC0(p, t)
            const float w = __fmul_rn(c, 0.0625f);
#pragma unroll
            for (int i = 0; i < 5; i++) acc[i] = __fmaf_rn(w, bk[i], acc[i]);
            if (lane == src) myc = c;
        }
        if (had) dp[o] = myc;
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int k = lane + 32 * i;
        if (k < 144) G1[(long long)p * 144 + k] = acc[i];
    }
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
        bx0 = min(bx0, __shfl_xor_sync(0xffffffffu, bx0, o2));
        by0 = min(by0, __shfl_xor_sync(0xffffffffu, by0, o2));
        bx1 = max(bx1, __shfl_xor_sync(0xffffffffu, bx1, o2));
        by1 = max(by1, __shfl_xor_sync(0xffffffffu, by1, o2));
    }
    if (lane == 0) box[p] = make_int4(bx0, by0, bx1, by1);
}

// Gim[t][k] = (1/16) sum over the patches p (ascending) and their pooled
// positions r (row-major) with argmax position t of c(p, r) * a_p[k], c the
// coefficients left by k_adj_g1_sparse -- the transposed product dC0^T * A
// restricted to the nonzeros of dC0.  One warp per segment of GSEG positions
// (tx0 .. tx0+GSEG-1, ty) of I': the pooled outputs that can point into it
// are rows ty>>1 .. (ty+1)>>1 and columns tx0/2 .. tx0/2+15 (lanes 0-15: the
// first row, 16-31: the second).  The warp finds, 32 boxes at a time, the
// patches whose box meets the segment, reads their candidate outputs, and
// adds each hit's c * a_p into the segment's [GSEG][144] accumulator in
// shared memory (lane j owns k = j + 32 i): a fixed order per position.
constexpr int GSEG = 30;
constexpr int GIM_WARPS = 2;

__global__ void __launch_bounds__(32 * GIM_WARPS) k_adj_gim(DmGeom g, const float* __restrict__ cP,
                                                           const unsigned char* __restrict__ amax0,
                                                           const int4* __restrict__ box, const float* __restrict__ Am,
                                                           float* __restrict__ Gim, int n_seg) {
    __shared__ float gs[GIM_WARPS][GSEG * 144];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int seg = blockIdx.x * GIM_WARPS + warp;
    if (seg >= n_seg) return;   // (no block-wide barrier below)
    const int W2 = g.W2, n0 = g.npatch(0);
    const int sxn = (W2 + GSEG - 1) / GSEG;
    const int tx0 = (seg % sxn) * GSEG, ty = seg / sxn;
    const int tx1 = min(tx0 + GSEG, W2) - 1;
    float* G = gs[warp];
    for (int i = lane; i < GSEG * 144; i += 32) G[i] = 0.0f;
    const int pw = g.dw[1], ph = g.dh[1];
    const long long psz = g.psize(1);
    const int ry = (ty >> 1) + (lane >> 4), rx = tx0 / 2 + (lane & 15);
    const bool cand = ry <= ((ty + 1) >> 1) && ry < ph && rx < pw;
    const long long off = (long long)ry * g.pitch(1) + rx;
    for (int pb = 0; pb < n0; pb += 32) {
        bool meets = false;
        if (pb + lane < n0) {
            const int4 bb = __ldg(box + pb + lane);
            meets = bb.x <= tx1 && bb.z >= tx0 && bb.y <= ty && bb.w >= ty;
        }
        unsigned int m = __ballot_sync(0xffffffffu, meets);
        while (m) {
            // up to four meeting patches at a time, their candidate outputs
            // loaded together, then taken in patch order
            int q[4], nq = 0;
            while (m && nq < 4) {
                q[nq++] = pb + __ffs(m) - 1;
                m &= m - 1;
            }
            float cv[4];
            int code[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                cv[j] = 0.0f;
                code[j] = 0;
                if (j < nq && cand) {
                    cv[j] = cP[(long long)q[j] * psz + off];
                    code[j] = amax0[(long long)q[j] * psz + off];
                }
            }
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (j >= nq) break;
                int tl = -1;
                if (cv[j] != 0.0f) {
                    const int tx = 2 * rx + code[j] % 3 - 1, tyy = 2 * ry + code[j] / 3 - 1;
                    if (tyy == ty && tx >= tx0 && tx <= tx1) tl = tx - tx0;
                }
                unsigned int h = __ballot_sync(0xffffffffu, tl >= 0);
                if (!h) continue;
                float a[5];
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    const int k = lane + 32 * i;
                    a[i] = k < 144 ? __ldg(Am + (long long)q[j] * 144 + k) : 0.0f;
                }
                while (h) {
                    const int src = __ffs(h) - 1;
                    h &= h - 1;
                    const float c = __shfl_sync(0xffffffffu, cv[j], src);
                    const int t = __shfl_sync(0xffffffffu, tl, src);
#pragma unroll
                    for (int i = 0; i < 5; i++) {
                        const int k = lane + 32 * i;
                        if (k < 144) G[t * 144 + k] = __fmaf_rn(c, a[i], G[t * 144 + k]);
                    }
                }
            }
        }
    }
    __syncwarp();
    for (int i = lane; i < GSEG * 144; i += 32) {
        const int tx = tx0 + i / 144;
        if (tx <= tx1) Gim[((long long)ty * W2 + tx) * 144 + i % 144] = __fmul_rn(0.0625f, G[i]);
    }
}

// g1[y][x][c] = G1[patch of (x, y)][(y%4*4 + x%4)*9 + c] (0 outside every atomic window).
__global__ void k_adj_g1(DmGeom g, const float* __restrict__ G1, float* __restrict__ g1) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.W1 * g.H1 * 9) return;
    const int ch = (int)(idx % 9);
    const long long pix = idx / 9;
    const int x = (int)(pix % g.W1), y = (int)(pix / g.W1);
    const int px = x / 4, py = y / 4;
    float v = 0.0f;
    if (px < g.P0x && py < g.P0y) v = G1[((long long)py * g.P0x + px) * 144 + ((y % 4) * 4 + (x % 4)) * 9 + ch];
    g1[idx] = v;
}

// g2[u][c] = sum over the 16 windows t = u + (2 - dx, 2 - dy) inside I' of Gim[t][(dy*4+dx)*9 + c].
__global__ void k_adj_g2(DmGeom g, const float* __restrict__ Gim, float* __restrict__ g2) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)g.W2 * g.H2 * 9) return;
    const int ch = (int)(idx % 9);
    const long long pix = idx / 9;
    const int x = (int)(pix % g.W2), y = (int)(pix / g.W2);
    float s = 0.0f;
    for (int dy = 0; dy < 4; dy++)
        for (int dx = 0; dx < 4; dx++) {
            const int tx = x + 2 - dx, ty = y + 2 - dy;
            if (tx < 0 || ty < 0 || tx >= g.W2 || ty >= g.H2) continue;
            s = __fadd_rn(s, Gim[((long long)ty * g.W2 + tx) * 144 + (dy * 4 + dx) * 9 + ch]);
        }
    g2[idx] = s;
}

inline unsigned nb(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void dm_grad_layout(const DmGeom& g, DmGradLayout* o) {
    memset(o, 0, sizeof(*o));
    size_t off = 0;
    o->parts = off; off = dm_align(off + (size_t)g.npatch(g.L) * 4);
    for (int l = 1; l <= g.L; l++) { o->dA[l] = off; off = dm_align(off + (size_t)g.npatch(l) * g.dsize(l) * 4); }
    for (int l = 0; l < g.L; l++) { o->dP[l] = off; off = dm_align(off + (size_t)g.npatch(l) * g.psize(l + 1) * 4); }
    const size_t T = (size_t)g.W2 * g.H2;
    o->Am = off; off = dm_align(off + (size_t)g.npatch(0) * 144 * 4);
    o->Bm = off; off = dm_align(off + T * 144 * 4);
    o->G1 = off; off = dm_align(off + (size_t)g.npatch(0) * 144 * 4);
    o->Gim = off; off = dm_align(off + T * 144 * 4);
    o->box = off; off = dm_align(off + (size_t)g.npatch(0) * sizeof(int4));
    for (int l = 1; l <= g.L; l++) { o->boxA[l] = off; off = dm_align(off + (size_t)g.npatch(l) * sizeof(int4)); }
    for (int l = 0; l < g.L; l++) { o->boxP[l] = off; off = dm_align(off + (size_t)g.npatch(l) * sizeof(int4)); }
    // children of any level: the atomic patches, or a lattice level (Lx x Ly >= P0x x P0y)
    const size_t nchild = (size_t)(g.npatch(0) > g.npatch(1) ? g.npatch(0) : g.npatch(1));
    o->par = off; off = dm_align(off + nchild * sizeof(int4));
    o->nch = off; off = dm_align(off + nchild * sizeof(int4));
    o->bytes = off;
}

cudaError_t dm_launch_loss_grad(const DmGeom& g, const dm_pyramid& py, const float* d1, const float* d2, float lam,
                                const DmGradLayout& gl, char* ws, float* d_loss, float* g1, float* g2, cudaStream_t st) {
    const int L = g.L;
    float* parts = reinterpret_cast<float*>(ws + gl.parts);
    long long launches = 0;
    auto boxA = [&](int l) { return reinterpret_cast<int4*>(ws + gl.boxA[l]); };
    auto boxP = [&](int l) { return reinterpret_cast<int4*>(ws + gl.boxP[l]); };
    int4* par = reinterpret_cast<int4*>(ws + gl.par);
    int4* nch = reinterpret_cast<int4*>(ws + gl.nch);
    k_adj_top<<<nb(g.npatch(L), 128), 128, 0, st>>>(g, py.valid[L], py.valid[L - 1], py.top, py.pooled[L - 1], lam,
                                                    py.compensated, reinterpret_cast<float*>(ws + gl.dA[L]), parts,
                                                    boxA(L));
    k_adj_loss<<<1, 256, 0, st>>>(parts, g.npatch(L), d_loss);
    launches += 2;
    if (!g1 || !g2) {   // loss only
        dm_count_launches(launches);
        return cudaGetLastError();
    }
    for (int l = L; l >= 1; l--) {
        const int np_child = g.npatch(l - 1);
        k_adj_box<<<nb(np_child, 128), 128, 0, st>>>(g, l, py.valid[l], py.valid[l - 1], boxA(l), boxP(l - 1),
                                                      l - 1 >= 1 ? boxA(l - 1) : nullptr, par, nch);
        dim3 grid(nb(g.dsize(l), 128 * ADJ_PPT), np_child);
        k_adj_pooled<<<grid, 128, 0, st>>>(g, l, reinterpret_cast<const float*>(ws + gl.dA[l]),
                                           reinterpret_cast<float*>(ws + gl.dP[l - 1]), boxA(l), boxP(l - 1), par, nch);
        launches += 2;
        if (l - 1 >= 1) {
            dim3 g2d(nb(g.dsize(l - 1), 128 * ADJ_PPT), g.npatch(l - 1));
            k_adj_unpool<<<g2d, 128, 0, st>>>(g, l - 1, py.valid[l - 1], py.valid[l - 2], py.pooled[l - 2],
                                              reinterpret_cast<const float*>(ws + gl.dP[l - 1]), py.amax[l - 1], lam,
                                              py.compensated, reinterpret_cast<float*>(ws + gl.dA[l - 1]), boxA(l - 1));
            launches++;
        }
    }
    float* Am = reinterpret_cast<float*>(ws + gl.Am);
    float* Bm = reinterpret_cast<float*>(ws + gl.Bm);
    float* G1 = reinterpret_cast<float*>(ws + gl.G1);
    float* Gim = reinterpret_cast<float*>(ws + gl.Gim);
    int4* box = reinterpret_cast<int4*>(ws + gl.box);
    float* dP0 = reinterpret_cast<float*>(ws + gl.dP[0]);
    const long long n0 = g.npatch(0), T = (long long)g.W2 * g.H2;
    k_adj_im2col<<<nb((n0 + T) * 144, 256), 256, 0, st>>>(g, d1, d2, Am, Bm);
    k_adj_g1_sparse<<<nb(n0, 8), 256, 0, st>>>(g, dP0, py.amax[0], Am, Bm, lam, G1, box, boxP(0));
    const long long n_seg = (long long)((g.W2 + GSEG - 1) / GSEG) * g.H2;
    k_adj_gim<<<nb(n_seg, GIM_WARPS), 32 * GIM_WARPS, 0, st>>>(g, dP0, py.amax[0], box, Am, Gim, (int)n_seg);
    launches += 3;
    k_adj_g1<<<nb((long long)g.W1 * g.H1 * 9, 256), 256, 0, st>>>(g, G1, g1);
    k_adj_g2<<<nb(T * 9, 256), 256, 0, st>>>(g, Gim, g2);
    launches += 2;
    dm_count_launches(launches);
    return cudaGetLastError();
}
