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
// G1 is a gather over the nonzeros of dC0 (at most one per pooled output),
// one warp per patch; Gim is a dense FP32 GEMM over chunks of patches (the
// dense dC0 block of a chunk is the only large temporary).  Then G1 is
// scattered onto the atomic windows of I and Gim gathered (col2im) onto the
// pixels of I'.
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
                          float* __restrict__ dA, float* __restrict__ parts) {
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

// dP_{l-1}(c, r) = sum over the parents p_i = c - 2^l o_i of c (i = 0..3, in
// order) of dA_l(p_i, r - o_i) / n(p_i).  Grid: (positions of domain l, child).
__global__ void k_adj_pooled(DmGeom g, int l, const unsigned char* __restrict__ vcur,
                             const unsigned char* __restrict__ vprev, const float* __restrict__ dA,
                             float* __restrict__ dP) {
    const int c = blockIdx.y;
    const int mw = g.dw[l], mh = g.dh[l], pitch = g.pitch(l);
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= mw * mh) return;
    const int rx = r % mw, ry = r / mw;
    float sum = 0.0f;
    if (vprev[c]) {
        const int cx = l == 1 ? c % g.P0x : c % g.Lx, cy = l == 1 ? c / g.P0x : c / g.Lx;
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
            int ix, iy;
            if (l == 1) { ix = cx + (1 - ox) / 2; iy = cy + (1 - oy) / 2; }
            else { const int s = 1 << (l - 2); ix = cx - ox * s; iy = cy - oy * s; }
            if (ix < 0 || iy < 0 || ix >= g.Lx || iy >= g.Ly) continue;
            const int p = iy * g.Lx + ix;
            if (!vcur[p]) continue;
            const int qx = rx - ox, qy = ry - oy;
            if (qx < 0 || qy < 0 || qx >= mw || qy >= mh) continue;
            int n = 0;
            for (int j = 0; j < 4; j++) {
                int cj = dm_child(g, l, ix, iy, j);
                if (cj >= 0 && vprev[cj]) n++;
            }
            const float d = dA[((long long)p * mh + qy) * mw + qx];
            if (d != 0.0f) sum = __fadd_rn(sum, __fdiv_rn(d, (float)n));
        }
    }
    dP[(long long)c * g.psize(l) + (long long)ry * pitch + rx] = sum;
}

// dA_{m}(c, t) for m = l-1 >= 1: sum over the pooled positions r whose argmax
// is t (r = floor/ceil(t/2) per axis, ascending) of dP_m(c, r) * lam A^(lam-1),
// A the unrectified average at t.  Grid: (positions of domain m, patch).
__global__ void k_adj_unpool(DmGeom g, int m, const unsigned char* __restrict__ vm, const unsigned char* __restrict__ vprev,
                             const float* __restrict__ prev, const float* __restrict__ dP,
                             const unsigned char* __restrict__ amax, float lam, int comp, float* __restrict__ dA) {
    const int c = blockIdx.y;
    const int tw = g.dw[m], th = g.dh[m];
    const int pw = g.dw[m + 1], ph = g.dh[m + 1], pitch = g.pitch(m + 1);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tw * th) return;
    const int tx = t % tw, ty = t / tw;
    float sum = 0.0f;
    if (vm[c]) {
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
// It also writes the same coefficients into row p - p0 of the dense dC0 block
// of patches [p0, p0 + pc) (zeroed before), added in the same order where two
// pooled positions share an argmax position, for the other product.
__global__ void __launch_bounds__(256) k_adj_g1_sparse(DmGeom g, int p0, int pc, const float* __restrict__ dP0,
                                                      const unsigned char* __restrict__ amax0,
                                                      const float* __restrict__ Am, const float* __restrict__ Bm,
                                                      float lam, float* __restrict__ G1, float* __restrict__ dC) {
    const int lane = threadIdx.x & 31;
    const int pl = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (pl >= pc) return;
    const int p = p0 + pl;
    float* dcrow = dC + (long long)pl * g.W2 * g.H2;
    const int pw = g.dw[1], ph = g.dh[1], pitch = g.pitch(1), W2 = g.W2;
    const float* dp = dP0 + (long long)p * g.psize(1);
    const unsigned char* am = amax0 + (long long)p * g.psize(1);
    float a[5], acc[5];
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int k = lane + 32 * i;
        a[i] = k < 144 ? __ldg(Am + (long long)p * 144 + k) : 0.0f;
        acc[i] = 0.0f;
    }
    const int n = pw * ph;
    for (int r0 = 0; r0 < n; r0 += 32) {
        const int r = r0 + lane;
        float d = 0.0f;
        int t = 0;
        if (r < n) {
            const int rx = r % pw, ry = r / pw;
            d = dp[(long long)ry * pitch + rx];
            if (d != 0.0f) {
                const int code = am[(long long)ry * pitch + rx];
                const int tx = 2 * rx + code % 3 - 1, ty = 2 * ry + code / 3 - 1;
                // (the forward's pooling only ever points inside I')
                if (code <= 8 && tx >= 0 && ty >= 0 && tx < W2 && ty < g.H2) t = ty * W2 + tx;
                else d = 0.0f;
            }
        }
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
            for (int o = 16; o > 0; o >>= 1) part = __fadd_rn(part, __shfl_xor_sync(0xffffffffu, part, o));
            const float c = __fmul_rn(dv, dpow(__fmul_rn(part, 0.0625f), lam));   // this r's share of dC0(p, t)
            const float w = __fmul_rn(c, 0.0625f);
#pragma unroll
            for (int i = 0; i < 5; i++) acc[i] = __fmaf_rn(w, bk[i], acc[i]);
            if (lane == 0) dcrow[tv] = __fadd_rn(dcrow[tv], c);
        }
    }
#pragma unroll
    for (int i = 0; i < 5; i++) {
        const int k = lane + 32 * i;
        if (k < 144) G1[(long long)p * 144 + k] = acc[i];
    }
}

// C[m][n] (+)= alpha * sum_k A[k][m] B[k][n] for n < 144: the transposed
// product of the level-0 backward (m = position of I', k = patch, n = the 144
// window entries).  128 x 144 tiles, K steps of 16, 256 threads, each 8 rows
// (m = 8 tm ..) x 9 columns (n = tn + 16 j) of the tile, the next K step's
// tiles prefetched into registers while the current one is multiplied.
__global__ void __launch_bounds__(256, 2) k_sgemm_tn144(int M, int K, float alpha, const float* __restrict__ A, long long lda,
                                                    const float* __restrict__ B, float* __restrict__ C, int accum) {
    constexpr int BM = 128, BN = 144, BK = 16;
    __shared__ __align__(16) float As[BK][BM];
    __shared__ float Bs[BK][BN];
    const int m0 = blockIdx.x * BM;
    const int tid = threadIdx.x;
    const int tm = tid >> 4, tn = tid & 15;
    float acc[8][9] = {};
    float ra[8], rb[9];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int idx = tid + 256 * e, kk = idx >> 7, mm = idx & 127;
            const int gm = m0 + mm, gk = k0 + kk;
            ra[e] = (gm < M && gk < K) ? __ldg(A + (long long)gk * lda + gm) : 0.0f;
        }
#pragma unroll
        for (int e = 0; e < 9; e++) {
            const int idx = tid + 256 * e, kk = idx / BN, nn = idx % BN;
            const int gk = k0 + kk;
            rb[e] = gk < K ? __ldg(B + (long long)gk * BN + nn) : 0.0f;
        }
    };
    auto stash = [&]() {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const int idx = tid + 256 * e;
            As[idx >> 7][idx & 127] = ra[e];
        }
#pragma unroll
        for (int e = 0; e < 9; e++) {
            const int idx = tid + 256 * e;
            Bs[idx / BN][idx % BN] = rb[e];
        }
    };
    fetch(0);
    for (int k0 = 0; k0 < K; k0 += BK) {
        stash();
        __syncthreads();
        if (k0 + BK < K) fetch(k0 + BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][8 * tm]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][8 * tm + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            float bv[9];
#pragma unroll
            for (int j = 0; j < 9; j++) bv[j] = Bs[kk][tn + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 9; j++) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; i++) {
        const int gm = m0 + 8 * tm + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 9; j++) {
            float* o = C + (long long)gm * BN + tn + 16 * j;
            const float v = __fmul_rn(alpha, acc[i][j]);
            *o = accum ? __fadd_rn(*o, v) : v;
        }
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
    // dense dC0 block of one chunk of patches: at most 1 GiB, at least one patch
    size_t pc = (size_t)1 << 30;
    pc /= (T * 4);
    if (pc < 1) pc = 1;
    if (pc > (size_t)g.npatch(0)) pc = (size_t)g.npatch(0);
    o->chunk = (int)pc;
    o->dC = off; off = dm_align(off + pc * T * 4);
    o->bytes = off;
}

cudaError_t dm_launch_loss_grad(const DmGeom& g, const dm_pyramid& py, const float* d1, const float* d2, float lam,
                                const DmGradLayout& gl, char* ws, float* d_loss, float* g1, float* g2, cudaStream_t st) {
    const int L = g.L;
    float* parts = reinterpret_cast<float*>(ws + gl.parts);
    long long launches = 0;
    k_adj_top<<<nb(g.npatch(L), 128), 128, 0, st>>>(g, py.valid[L], py.valid[L - 1], py.top, py.pooled[L - 1], lam,
                                                    py.compensated, reinterpret_cast<float*>(ws + gl.dA[L]), parts);
    k_adj_loss<<<1, 256, 0, st>>>(parts, g.npatch(L), d_loss);
    launches += 2;
    if (!g1 || !g2) {   // loss only
        dm_count_launches(launches);
        return cudaGetLastError();
    }
    for (int l = L; l >= 1; l--) {
        const int np_child = g.npatch(l - 1);
        dim3 grid(nb(g.dsize(l), 128), np_child);
        k_adj_pooled<<<grid, 128, 0, st>>>(g, l, py.valid[l], py.valid[l - 1], reinterpret_cast<const float*>(ws + gl.dA[l]),
                                           reinterpret_cast<float*>(ws + gl.dP[l - 1]));
        launches++;
        if (l - 1 >= 1) {
            dim3 g2d(nb(g.dsize(l - 1), 128), g.npatch(l - 1));
            k_adj_unpool<<<g2d, 128, 0, st>>>(g, l - 1, py.valid[l - 1], py.valid[l - 2], py.pooled[l - 2],
                                              reinterpret_cast<const float*>(ws + gl.dP[l - 1]), py.amax[l - 1], lam,
                                              py.compensated, reinterpret_cast<float*>(ws + gl.dA[l - 1]));
            launches++;
        }
    }
    float* Am = reinterpret_cast<float*>(ws + gl.Am);
    float* Bm = reinterpret_cast<float*>(ws + gl.Bm);
    float* G1 = reinterpret_cast<float*>(ws + gl.G1);
    float* Gim = reinterpret_cast<float*>(ws + gl.Gim);
    float* dC = reinterpret_cast<float*>(ws + gl.dC);
    const long long n0 = g.npatch(0), T = (long long)g.W2 * g.H2;
    k_adj_im2col<<<nb((n0 + T) * 144, 256), 256, 0, st>>>(g, d1, d2, Am, Bm);
    launches++;
    for (long long p0 = 0; p0 < n0; p0 += gl.chunk) {
        const int pc = (int)(n0 - p0 < gl.chunk ? n0 - p0 : gl.chunk);
        // the chunk's dC0 rows and G1 rows from the nonzeros of dC0
        cudaError_t e = cudaMemsetAsync(dC, 0, (size_t)pc * T * sizeof(float), st);
        if (e != cudaSuccess) return e;
        k_adj_g1_sparse<<<nb(pc, 8), 256, 0, st>>>(g, (int)p0, pc, reinterpret_cast<const float*>(ws + gl.dP[0]),
                                                   py.amax[0], Am, Bm, lam, G1, dC);
        // Gim (+)= (1/16) dC^T [T x pc] * Am[p0 .. p0+pc) [pc x 144]
        k_sgemm_tn144<<<nb(T, 128), 256, 0, st>>>((int)T, pc, 0.0625f, dC, T, Am + p0 * 144, Gim, p0 != 0);
        launches += 2;
    }
    k_adj_g1<<<nb((long long)g.W1 * g.H1 * 9, 256), 256, 0, st>>>(g, G1, g1);
    k_adj_g2<<<nb(T * 9, 256), 256, 0, st>>>(g, Gim, g2);
    launches += 2;
    dm_count_launches(launches);
    return cudaGetLastError();
}
