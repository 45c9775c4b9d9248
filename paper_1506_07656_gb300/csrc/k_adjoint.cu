// Differentiable form: loss = sum over existing top patches p of
// max_q C_L(p, q) (first maximum), and its gradient with respect to both
// descriptor fields (the paper has no loss; this is the adjoint of
// Algorithm 1).  The backward runs through
//   the rectification  C = A^lambda                  (Eq. 11),
//   the shifted average A_l = mean_i P_{l-1}(c_i, q+o_i)   (Eq. 12),
//   the max-pooling with its saved argmax            (Eq. 8-9),
//   the level-0 correlation C0 = (1/16) a_p . b_t    (Eq. 3-4).
// Every value is a gather with a fixed summation order, so the gradient is
// deterministic.  Per level two dense arrays hold the values: dA_l on the
// map domain of level l (unrectified averages) and dP_l in the pooled layout,
// zero outside the gradient's support; only the support is visited: the
// nonzeros of each array are listed (a frontier, as in the backtracking) and
// the next array's entries are found from them, each one computed once by
// its fixed-order gather and claimed by an atomic compare-and-swap on its
// (zero) slot, so that a value several frontier items reach is written and
// listed once.
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
// dA_L = d(A^lam)/dA at that position (zero elsewhere), listed in E.
__global__ void k_adj_top(DmGeom g, const unsigned char* __restrict__ vL, const unsigned char* __restrict__ vprev,
                          const float* __restrict__ top, const float* __restrict__ prev, float lam, int comp,
                          float* __restrict__ dA, float* __restrict__ parts, int2* __restrict__ E,
                          unsigned int* __restrict__ nE) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const int L = g.L;
    if (p >= g.npatch(L)) return;
    const int nq = g.dw[L] * g.dh[L];
    float* d = dA + (long long)p * nq;
    for (int q = 0; q < nq; q++) d[q] = 0.0f;
    if (!vL[p]) { parts[p] = 0.0f; return; }
    const float* t = top + (long long)p * nq;
    float best = -INFINITY;
    int qb = 0;
    for (int q = 0; q < nq; q++)
        if (t[q] > best) { best = t[q]; qb = q; }
    parts[p] = best;
    int n;
    const float a = level_average(g, L, p, qb % g.dw[L], qb / g.dw[L], vprev, prev, comp != 0, &n);
    d[qb] = dpow(a, lam);
    if (d[qb] != 0.0f) E[atomicAdd(nE, 1u)] = make_int2(p, qb);   // at most npatch(L) entries
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

// Claim the zero slot of a nonzero value: true for the one caller that wrote
// it (every caller computes the same bits by the same fixed-order gather).
__device__ __forceinline__ bool claim(float* slot, float v) {
    return atomicCAS(reinterpret_cast<unsigned int*>(slot), 0u, __float_as_uint(v)) == 0u;
}

// One step down from level l.  For every nonzero dA_l(p, q) of the frontier E
// and every child slot i of p: the pooled position r = q + o_i of child c_i
// at level l - 1, and there
//   dP_{l-1}(c, r) = sum over the parents p_j = c - 2^l o_j of c (j = 0..3, in
//   order) of dA_l(p_j, r - o_j) / n(p_j)
// (every nonzero dP is reached: one of its terms is a listed dA).  Claimed
// entries are listed in F, or, at l = 1, folded into the box of each atomic
// patch's nonzeros (x0, y0, -x1, -y1 by atomic minima).  Work item w = 4e + i,
// grid-stride over the frontier's count.
__global__ void __launch_bounds__(256) k_adj_down(DmGeom g, int l, const unsigned char* __restrict__ vcur,
                                                  const unsigned char* __restrict__ vprev, const float* __restrict__ dA,
                                                  float* __restrict__ dP, const int2* __restrict__ E,
                                                  const unsigned int* __restrict__ nE, int2* __restrict__ F,
                                                  unsigned int* __restrict__ nF, unsigned int capF,
                                                  unsigned int* __restrict__ overflow, int* __restrict__ box0) {
    const unsigned long long n = 4ull * min(*nE, capF);   // (E and F share one capacity)
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const int2 e = E[w >> 2];
        const int i = (int)(w & 3u);
        const int p = e.x, qx = e.y % mw, qy = e.y / mw;
        const int c = dm_child(g, l, p % g.Lx, p / g.Lx, i);
        if (c < 0 || !vprev[c]) continue;
        const int rx = qx + ((i >= 2) ? 1 : -1), ry = qy + ((i & 1) ? 1 : -1);
        if (rx < 0 || ry < 0 || rx >= mw || ry >= mh) continue;
        float sum = 0.0f;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int nj;
            const int pj = adj_parent(g, l, c, j, vcur, vprev, &nj);
            if (pj < 0) continue;
            const int sx = rx - ((j >= 2) ? 1 : -1), sy = ry - ((j & 1) ? 1 : -1);
            if (sx < 0 || sy < 0 || sx >= mw || sy >= mh) continue;
            const float d = dA[((long long)pj * mh + sy) * mw + sx];
            if (d != 0.0f) sum = __fadd_rn(sum, __fdiv_rn(d, (float)nj));
        }
        if (sum == 0.0f) continue;
        if (!claim(dP + (long long)c * g.psize(l) + (long long)ry * pitch + rx, sum)) continue;
        if (box0) {
            atomicMin(box0 + 4 * c, rx);
            atomicMin(box0 + 4 * c + 1, ry);
            atomicMin(box0 + 4 * c + 2, -rx);
            atomicMin(box0 + 4 * c + 3, -ry);
        } else {
            const unsigned int k = atomicAdd(nF, 1u);
            if (k < capF) F[k] = make_int2(c, ry * mw + rx);
            else atomicOr(overflow, 1u);
        }
    }
}

// One step up to the map domain of level m = l - 1 >= 1.  For every nonzero
// dP_m(c, r) of the frontier F: its argmax position t = 2r + (m_x, m_y), and
// there
//   dA_m(c, t) = (sum over the pooled positions r' whose argmax is t, r' =
//   floor/ceil(t/2) per axis ascending, of dP_m(c, r')) * lam A^(lam-1),
// A the unrectified average at t.  Claimed entries are listed in E.
__global__ void __launch_bounds__(256) k_adj_up(DmGeom g, int m, const unsigned char* __restrict__ vm,
                                                const unsigned char* __restrict__ vprev,
                                                const float* __restrict__ prev, const float* __restrict__ dP,
                                                const unsigned char* __restrict__ amax, float lam, int comp,
                                                float* __restrict__ dA, const int2* __restrict__ F,
                                                const unsigned int* __restrict__ nF, int2* __restrict__ E,
                                                unsigned int* __restrict__ nE, unsigned int capE,
                                                unsigned int* __restrict__ overflow) {
    const unsigned long long n = min(*nF, capE);   // (E and F share one capacity)
    const int tw = g.dw[m], th = g.dh[m];
    const int pw = g.dw[m + 1], ph = g.dh[m + 1], pitch = g.pitch(m + 1);
    const long long psz = g.psize(m + 1);
    for (unsigned long long w = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; w < n;
         w += (unsigned long long)gridDim.x * blockDim.x) {
        const int2 f = F[w];
        const int c = f.x, r0x = f.y % pw, r0y = f.y / pw;
        if (!vm[c]) continue;
        const int code0 = amax[c * psz + (long long)r0y * pitch + r0x];
        if (code0 > 8) continue;   // (the forward's pooling never writes one)
        const int tx = 2 * r0x + code0 % 3 - 1, ty = 2 * r0y + code0 / 3 - 1;
        if (tx < 0 || ty < 0 || tx >= tw || ty >= th) continue;
        float dsum = 0.0f;
        for (int ry = ty >> 1; ry <= (ty + 1) >> 1; ry++) {
            if (ry >= ph) continue;
            for (int rx = tx >> 1; rx <= (tx + 1) >> 1; rx++) {
                if (rx >= pw) continue;
                const long long o = c * psz + (long long)ry * pitch + rx;
                const int code = amax[o];
                if (2 * rx + code % 3 - 1 != tx || 2 * ry + code / 3 - 1 != ty) continue;
                dsum = __fadd_rn(dsum, dP[o]);
            }
        }
        if (dsum == 0.0f) continue;
        int nn;
        const float a = level_average(g, m, c, tx, ty, vprev, prev, comp != 0, &nn);
        const float v = __fmul_rn(dsum, dpow(a, lam));
        if (v == 0.0f) continue;
        if (!claim(dA + ((long long)c * th + ty) * tw + tx, v)) continue;
        const unsigned int k = atomicAdd(nE, 1u);
        if (k < capE) E[k] = make_int2(c, ty * tw + tx);
        else atomicOr(overflow, 1u);
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
// Only the box of the nonzeros of dP0 is scanned (boxP0[p] = (x0, y0, -x1, -y1)
// from k_adj_down; x0 > x1 when the patch has none).
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
    const int4 sbn = boxP0[p];
    const int4 sb = make_int4(sbn.x, sbn.y, -sbn.z, -sbn.w);
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
            // up to two nonzeros at a time: their windows of I' loaded together,
            // then taken in order
            int src[2];
            src[0] = __ffs(nz) - 1;
            nz &= nz - 1;
            src[1] = nz ? __ffs(nz) - 1 : -1;
            if (nz) nz &= nz - 1;
            float bk[2][5];
#pragma unroll
            for (int u = 0; u < 2; u++) {
                const int tv = __shfl_sync(0xffffffffu, t, src[u] < 0 ? 0 : src[u]);
                const float* b = Bm + (long long)tv * 144;
#pragma unroll
                for (int i = 0; i < 5; i++) {
                    const int k = lane + 32 * i;
                    bk[u][i] = (src[u] >= 0 && k < 144) ? __ldg(b + k) : 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < 2; u++) {
                if (src[u] < 0) break;
                const float dv = __shfl_sync(0xffffffffu, d, src[u]);
                float part = 0.0f;
#pragma unroll
                for (int i = 0; i < 5; i++) part = __fmaf_rn(a[i], bk[u][i], part);
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o2));
                const float c = __fmul_rn(dv, dpow(__fmul_rn(part, 0.0625f), lam));   // this r's share of dC0(p, t)
                const float w = __fmul_rn(c, 0.0625f);
#pragma unroll
                for (int i = 0; i < 5; i++) acc[i] = __fmaf_rn(w, bk[u][i], acc[i]);
                if (lane == src[u]) myc = c;
            }
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
    int4 nb4 = lane < n0 ? __ldg(box + lane) : make_int4(0, 0, -1, -1);
    for (int pb = 0; pb < n0; pb += 32) {
        const int4 bb = nb4;   // this chunk's boxes; the next chunk's are loaded meanwhile
        nb4 = pb + 32 + lane < n0 ? __ldg(box + pb + 32 + lane) : make_int4(0, 0, -1, -1);
        const bool meets = bb.x <= tx1 && bb.z >= tx0 && bb.y <= ty && bb.w >= ty;
        unsigned int m = __ballot_sync(0xffffffffu, meets);
        while (m) {
            // up to eight meeting patches at a time, their candidate outputs
            // loaded together, then taken in patch order
            int q[8], nq = 0;
            while (m && nq < 8) {
                q[nq++] = pb + __ffs(m) - 1;
                m &= m - 1;
            }
            float cv[8];
            int code[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                cv[j] = 0.0f;
                code[j] = 0;
                if (j < nq && cand) {
                    cv[j] = cP[(long long)q[j] * psz + off];
                    code[j] = amax0[(long long)q[j] * psz + off];
                }
            }
#pragma unroll
            for (int j = 0; j < 8; j++) {
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
    o->box0 = off; off = dm_align(off + (size_t)g.npatch(0) * sizeof(int4));
    // frontiers: E_l (nonzeros of dA_l, l >= 1) and F_l (nonzeros of dP_l, l >= 1;
    // F_0 is folded into box0).  A frontier at level l holds at most
    // 4^(L-l) npatch(L) entries (each step down has 4 children per entry, each
    // step up one argmax per entry) and at most its array's size.
    size_t cap = 0;
    for (int l = 1; l <= g.L; l++) {
        size_t tree = (size_t)g.npatch(g.L);
        for (int k = l; k < g.L && tree < ((size_t)1 << 40); k++) tree *= 4;
        const size_t eA = (size_t)g.npatch(l) * g.dsize(l);
        const size_t eP = l < g.L ? (size_t)g.npatch(l) * g.dw[l + 1] * g.dh[l + 1] : 0;
        cap = std::max(cap, std::min(tree, std::max(eA, eP)));
    }
    o->cap_ok = cap <= (size_t)0xffffffffu;   // frontier counts are 32-bit
    cap = std::min(cap, (size_t)0xffffffffu);
    o->cap = (unsigned int)cap;
    o->frontE = off; off = dm_align(off + cap * sizeof(int2));
    o->frontF = off; off = dm_align(off + cap * sizeof(int2));
    o->counts = off; off = dm_align(off + (size_t)DM_GRAD_COUNTS * sizeof(unsigned int));
    o->bytes = off;
}

cudaError_t dm_launch_loss_grad(const DmGeom& g, const dm_pyramid& py, const float* d1, const float* d2, float lam,
                                const DmGradLayout& gl, char* ws, float* d_loss, float* g1, float* g2, cudaStream_t st) {
    const int L = g.L;
    float* parts = reinterpret_cast<float*>(ws + gl.parts);
    long long launches = 0;
    if (!gl.cap_ok) return cudaErrorInvalidValue;
    int2* E = reinterpret_cast<int2*>(ws + gl.frontE);
    int2* F = reinterpret_cast<int2*>(ws + gl.frontF);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + gl.counts);   // [2l]: E_l, [2l+1]: F_l, last: overflow
    unsigned int* overflow = cnt + DM_GRAD_COUNTS - 1;
    int* box0 = reinterpret_cast<int*>(ws + gl.box0);
    cudaError_t em = cudaMemsetAsync(cnt, 0, DM_GRAD_COUNTS * sizeof(unsigned int), st);
    if (em != cudaSuccess) return em;
    k_adj_top<<<nb(g.npatch(L), 128), 128, 0, st>>>(g, py.valid[L], py.valid[L - 1], py.top, py.pooled[L - 1], lam,
                                                    py.compensated, reinterpret_cast<float*>(ws + gl.dA[L]), parts,
                                                    E, cnt + 2 * L);
    k_adj_loss<<<1, 256, 0, st>>>(parts, g.npatch(L), d_loss);
    launches += 2;
    if (!g1 || !g2) {   // loss only
        dm_count_launches(launches);
        return cudaGetLastError();
    }
    // the dense arrays below level L start at zero: the frontier kernels write
    // only the support (dA_L itself is written whole by k_adj_top)
    if (L >= 2) {
        em = cudaMemsetAsync(ws + gl.dA[1], 0, gl.dA[L] - gl.dA[1], st);
        if (em != cudaSuccess) return em;
    }
    em = cudaMemsetAsync(ws + gl.dP[0], 0, gl.dP[L - 1] + (size_t)g.npatch(L - 1) * g.psize(L) * 4 - gl.dP[0], st);
    if (em == cudaSuccess) em = cudaMemsetAsync(box0, 0x7f, (size_t)g.npatch(0) * sizeof(int4), st);
    if (em != cudaSuccess) return em;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned int fgrid = (unsigned int)nsm * 8;
    for (int l = L; l >= 1; l--) {
        k_adj_down<<<fgrid, 256, 0, st>>>(g, l, py.valid[l], py.valid[l - 1], reinterpret_cast<const float*>(ws + gl.dA[l]),
                                          reinterpret_cast<float*>(ws + gl.dP[l - 1]), E, cnt + 2 * l, F,
                                          cnt + 2 * (l - 1) + 1, gl.cap, overflow, l == 1 ? box0 : nullptr);
        launches++;
        if (l - 1 >= 1) {
            k_adj_up<<<fgrid, 256, 0, st>>>(g, l - 1, py.valid[l - 1], py.valid[l - 2], py.pooled[l - 2],
                                            reinterpret_cast<const float*>(ws + gl.dP[l - 1]), py.amax[l - 1], lam,
                                            py.compensated, reinterpret_cast<float*>(ws + gl.dA[l - 1]), F,
                                            cnt + 2 * (l - 1) + 1, E, cnt + 2 * (l - 1), gl.cap, overflow);
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
    k_adj_g1_sparse<<<nb(n0, 8), 256, 0, st>>>(g, dP0, py.amax[0], Am, Bm, lam, G1, box,
                                               reinterpret_cast<const int4*>(box0));
    const long long n_seg = (long long)((g.W2 + GSEG - 1) / GSEG) * g.H2;
    k_adj_gim<<<nb(n_seg, GIM_WARPS), 32 * GIM_WARPS, 0, st>>>(g, dP0, py.amax[0], box, Am, Gim, (int)n_seg);
    launches += 3;
    k_adj_g1<<<nb((long long)g.W1 * g.H1 * 9, 256), 256, 0, st>>>(g, G1, g1);
    k_adj_g2<<<nb(T * 9, 256), 256, 0, st>>>(g, Gim, g2);
    launches += 2;
    dm_count_launches(launches);
    return cudaGetLastError();
}
