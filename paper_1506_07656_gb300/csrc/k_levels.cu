// Pyramid levels l >= 1 (Eq. 5-12, boundary rule of Sec. 3.2, Algorithm 1).
//
// For a lattice patch p at level l with existing children c_i = p + 2^l o_i:
//   C_l(p, q) = (1/n) sum_{existing i} P_{l-1}(c_i, q + o_i)      (0 outside the domain)
// and, below the top, the stored pooled map
//   P_l(p, r) = (max over in-domain m of C_l(p, 2r + m))^lambda   + argmax code,
// or at the top C_L(p, q) = (C_l(p, q))^lambda.
// The children's sum is a compensated (TwoSum) sum in child order i = 0..3,
// rounded once and divided by n; pooling is on the unrectified average and the
// power is applied to the pooled value (x -> x^lambda is increasing on [0,1]).
//
// This pass is bound by HBM bandwidth: per stored output it reads the 4 child
// maps around 2r and writes 4 + 1 bytes.  Threads own one output each and
// consecutive threads consecutive rx, so each child-map row is read coalesced;
// the 3x3 windows of neighbouring outputs overlap and are served by L1/L2.
#include "dm_internal.cuh"

namespace {

// valid[l][p] = 1 iff some child exists (Eq. 7 with the boundary rule).
__global__ void k_valid(DmGeom g, int l, const unsigned char* __restrict__ vprev, unsigned char* __restrict__ v) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Lx * g.Ly) return;
    int ix = p % g.Lx, iy = p / g.Lx;
    unsigned char any = 0;
    for (int i = 0; i < 4; i++) {
        int c = dm_child(g, l, ix, iy, i);
        if (c >= 0 && vprev[c]) any = 1;
    }
    v[p] = any;
}

__global__ void k_fill_u8(unsigned char* p, int n, unsigned char val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = val;
}

struct Kids {
    const float* base[4];
    int n;
};

__device__ __forceinline__ float child_mean(const Kids& k, int qx, int qy, int mw, int mh) {
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (k.base[i] == nullptr) continue;
        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        int rx = qx + ox, ry = qy + oy;
        float v = 0.0f;
        if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) v = __ldg(k.base[i] + (long long)ry * mw + rx);
        float t = __fadd_rn(s, v);
        float bp = __fsub_rn(t, s);
        float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
        s = t;
        comp = __fadd_rn(comp, err);
    }
    return __fdiv_rn(__fadd_rn(s, comp), (float)k.n);
}

__device__ __forceinline__ bool load_kids(const DmGeom& g, int l, int p, const unsigned char* __restrict__ vprev,
                                          const float* __restrict__ prev, Kids& k) {
    int ix = p % g.Lx, iy = p / g.Lx;
    long long cs = (long long)g.dw[l] * g.dh[l];     // child pooled map size (domain of level l)
    k.n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int c = dm_child(g, l, ix, iy, i);
        if (c >= 0 && vprev[c]) {
            k.base[i] = prev + (long long)c * cs;
            k.n++;
        } else {
            k.base[i] = nullptr;
        }
    }
    return k.n > 0;
}

// Level l in [1, L-1]: pooled output P_l over the domain of level l+1.
__global__ void k_level_pool(DmGeom g, int l, const unsigned char* __restrict__ vprev,
                             const unsigned char* __restrict__ vcur, const float* __restrict__ prev,
                             float* __restrict__ out, unsigned char* __restrict__ amax, float lam) {
    const int p = blockIdx.y;
    if (!vcur[p]) return;
    const int ow = g.dw[l + 1], oh = g.dh[l + 1];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= ow * oh) return;
    const int rx = r % ow, ry = r / ow;
    const int mw = g.dw[l], mh = g.dh[l];
    Kids k;
    load_kids(g, l, p, vprev, prev, k);
    float best = -INFINITY;
    int code = 4;
#pragma unroll
    for (int my = -1; my <= 1; my++) {
#pragma unroll
        for (int mx = -1; mx <= 1; mx++) {
            int qx = 2 * rx + mx, qy = 2 * ry + my;
            if (qx < 0 || qy < 0 || qx >= mw || qy >= mh) continue;
            float a = child_mean(k, qx, qy, mw, mh);
            if (a > best) { best = a; code = (my + 1) * 3 + (mx + 1); }
        }
    }
    long long o = (long long)p * ow * oh + r;
    out[o] = dm_powf(best, lam);
    amax[o] = (unsigned char)code;
}

// Top level L: C_L = (mean of children)^lambda over the domain of level L.
__global__ void k_level_top(DmGeom g, int l, const unsigned char* __restrict__ vprev,
                            const unsigned char* __restrict__ vcur, const float* __restrict__ prev,
                            float* __restrict__ top, float lam) {
    const int p = blockIdx.y;
    if (!vcur[p]) return;
    const int mw = g.dw[l], mh = g.dh[l];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= mw * mh) return;
    Kids k;
    load_kids(g, l, p, vprev, prev, k);
    float a = child_mean(k, q % mw, q / mw, mw, mh);
    top[(long long)p * mw * mh + q] = dm_powf(a, lam);
}

}  // namespace

cudaError_t dm_launch_levels(const DmGeom& g, const dm_pyramid& py, float lam, cudaStream_t st) {
    const int B = 128;
    int n0 = g.npatch(0), np = g.npatch(1);
    k_fill_u8<<<(n0 + 255) / 256, 256, 0, st>>>(const_cast<unsigned char*>(py.valid[0]), n0, 1);
    for (int l = 1; l <= g.L; l++) {
        k_valid<<<(np + 255) / 256, 256, 0, st>>>(g, l, py.valid[l - 1], const_cast<unsigned char*>(py.valid[l]));
        if (l < g.L) {
            int n = g.dw[l + 1] * g.dh[l + 1];
            dim3 grid((n + B - 1) / B, np);
            k_level_pool<<<grid, B, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1],
                                              const_cast<float*>(py.pooled[l]),
                                              const_cast<unsigned char*>(py.amax[l]), lam);
        } else {
            int n = g.dw[l] * g.dh[l];
            dim3 grid((n + B - 1) / B, np);
            k_level_top<<<grid, B, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1],
                                             const_cast<float*>(py.top), lam);
        }
    }
    dm_count_launches(1 + 2 * g.L);
    return cudaGetLastError();
}
