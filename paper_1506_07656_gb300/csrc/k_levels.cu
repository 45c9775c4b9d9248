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
// This pass is bound by HBM bandwidth.  A CTA owns one patch and a tile of
// 32 x 8 pooled outputs: it stages the 4 child-map windows it needs (65 x 17
// values each, zero outside the domain) in shared memory with coalesced row
// loads, forms the 65 x 17 averages once, then pools them.  Patches vary
// fastest in the grid, so the (up to 4) parents that read the same child
// window run at about the same time and the repeat reads hit L2: HBM sees each
// child map about once.  Algorithmic bytes per stored output: 4 x 4 B of child
// values read (each child value feeds 4 outputs' worth of area) + 4 B + 1 B
// written.
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

constexpr int TW = 32, TH = 8;                 // pooled outputs per CTA (lane, warp)
constexpr int AW = 2 * TW + 1, AH = 2 * TH + 1;  // averages per CTA

// x / n rounded once, for n in 1..4: multiplications by 1, 1/2, 1/4 are exact,
// so they equal the correctly rounded quotient; n = 3 divides.
__device__ __forceinline__ float div_n(float x, int n) {
    return n == 3 ? __fdiv_rn(x, 3.0f) : __fmul_rn(x, n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.0f));
}

// Level l in [1, L-1], shared-memory tiled: grid (patch, tile), 8 warps.
// Rows of every staged window are spread over warps and columns over lanes,
// so each staged value costs one asynchronous 4-byte copy and a few integer
// operations (the previous per-element div/mod dominated the instruction count).
__global__ void __launch_bounds__(256) k_level_pool_tiled(DmGeom g, int l, const unsigned char* __restrict__ vprev,
                                                          const unsigned char* __restrict__ vcur,
                                                          const float* __restrict__ prev, float* __restrict__ out,
                                                          unsigned char* __restrict__ amax, float lam) {
    __shared__ float kid[4][AH][AW];
    __shared__ float avg[AH][AW];
    const int p = blockIdx.x;
    if (!vcur[p]) return;
    const int ow = g.dw[l + 1], oh = g.dh[l + 1];
    const int mw = g.dw[l], mh = g.dh[l];
    const int tiles_x = (ow + TW - 1) / TW;
    const int rx0 = (blockIdx.y % tiles_x) * TW, ry0 = (blockIdx.y / tiles_x) * TH;
    const int qx0 = 2 * rx0 - 1, qy0 = 2 * ry0 - 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Kids k;
    load_kids(g, l, p, vprev, prev, k);
    // Stage the child windows (child i is sampled at q + o_i); a source size of
    // 0 fills zeros outside the domain or for a missing child.
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        const float* base = k.base[i];
        for (int ay = warp; ay < AH; ay += 8) {
            const int ry = qy0 + ay + oy;
            const bool row_in = base != nullptr && ry >= 0 && ry < mh;
            const float* rowp = row_in ? base + (long long)ry * mw : prev;
            const unsigned dst0 = (unsigned)__cvta_generic_to_shared(&kid[i][ay][0]);
#pragma unroll
            for (int ax = lane; ax < AW; ax += 32) {
                const int rx = qx0 + ax + ox;
                const bool in = row_in && rx >= 0 && rx < mw;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                             :: "r"(dst0 + 4u * ax), "l"(in ? rowp + rx : prev), "r"(in ? 4 : 0) : "memory");
            }
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // averages: compensated sum over existing children in order i = 0..3, / n
    for (int ay = warp; ay < AH; ay += 8) {
#pragma unroll
        for (int ax = lane; ax < AW; ax += 32) {
            float s = 0.0f, comp = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (k.base[i] == nullptr) continue;
                float v = kid[i][ay][ax];
                float t = __fadd_rn(s, v);
                float bp = __fsub_rn(t, s);
                float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
                s = t;
                comp = __fadd_rn(comp, err);
            }
            avg[ay][ax] = div_n(__fadd_rn(s, comp), k.n);
        }
    }
    __syncthreads();
    // 3x3 / 2 max-pool over in-domain averages, first strict maximum, power
    const int rx = rx0 + lane, ry = ry0 + warp;
    if (rx >= ow || ry >= oh) return;
    float best = -INFINITY;
    int code = 4;
#pragma unroll
    for (int my = -1; my <= 1; my++) {
#pragma unroll
        for (int mx = -1; mx <= 1; mx++) {
            int qx = 2 * rx + mx, qy = 2 * ry + my;
            if (qx < 0 || qy < 0 || qx >= mw || qy >= mh) continue;
            float a = avg[2 * warp + 1 + my][2 * lane + 1 + mx];
            if (a > best) { best = a; code = (my + 1) * 3 + (mx + 1); }
        }
    }
    long long o = (long long)p * ow * oh + (long long)ry * ow + rx;
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
            int tiles = ((g.dw[l + 1] + TW - 1) / TW) * ((g.dh[l + 1] + TH - 1) / TH);
            dim3 grid(np, tiles);
            k_level_pool_tiled<<<grid, TW * TH, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1],
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
