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
// This pass streams the pooled maps of the level below (bandwidth) and does
// a fixed amount of arithmetic per stored output (4 compensated averages,
// a 9-way max with argmax, one power).  A CTA owns one patch and a tile of
// 32 x 16 pooled outputs (two per thread): it stages the 4 child-map windows
// it needs in shared memory with 16-byte asynchronous copies (rows of the
// pooled maps are padded to 8 floats, so every window row starts aligned; the
// copy's source size zero-fills whatever lies outside the domain), forms the
// 65 x 33 averages once, then pools them.  Patches vary fastest in the grid,
// so the (up to 4) parents that read the same child window run at about the
// same time and the repeat reads hit L2.  Algorithmic bytes per stored
// output: 16 B of child values read (each child value is shared by 4
// parents), 4 + 1 B written.
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

__device__ __forceinline__ float child_mean(const Kids& k, int qx, int qy, int mw, int mh, int pitch) {
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (k.base[i] == nullptr) continue;
        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
        int rx = qx + ox, ry = qy + oy;
        float v = 0.0f;
        if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) v = __ldg(k.base[i] + (long long)ry * pitch + rx);
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
    long long cs = g.psize(l);     // child pooled map size (domain of level l, padded rows)
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

constexpr int TW = 32, TH = 16;                // pooled outputs per CTA (lane, 2 x warp)
constexpr int AW = 2 * TW + 1, AH = 2 * TH + 1;  // averages per CTA (65 x 33)
constexpr int KW = 72;                           // staged child columns: 18 aligned float4
constexpr int AWP = 68;                          // padded row of the averages (16-byte aligned rows)
constexpr int LEVEL_THREADS = 256;

// x / n rounded once, for n in 1..4: multiplications by 1, 1/2, 1/4 are exact,
// so they equal the correctly rounded quotient; n = 3 divides.
__device__ __forceinline__ float div_n(float x, int n) {
    return n == 3 ? __fdiv_rn(x, 3.0f) : __fmul_rn(x, n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.0f));
}

// Knuth TwoSum step of the compensated child sum.
__device__ __forceinline__ void two_sum_add(float& s, float& comp, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    comp = __fadd_rn(comp, err);
}

// Average at staged position (ay, column c of child 0's frame) from the four
// child windows: child i contributes kid[i][ay][ax + ox_i + 3].
template <bool ALL4>
__device__ __forceinline__ float4 avg4(const float (*kid)[AH][KW], int ay, int ax, const int* ci, int n) {
    // children with ox = -1 (i = 0, 1) read columns ax+2 .. ax+5 (8-byte aligned),
    // children with ox = +1 (i = 2, 3) read columns ax+4 .. ax+7 (16-byte aligned)
    float v[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (!ALL4 && ci[i] < 0) continue;
        if (i < 2) {
            const float2 a = *reinterpret_cast<const float2*>(&kid[i][ay][ax + 2]);
            const float2 b = *reinterpret_cast<const float2*>(&kid[i][ay][ax + 4]);
            v[i][0] = a.x; v[i][1] = a.y; v[i][2] = b.x; v[i][3] = b.y;
        } else {
            const float4 a = *reinterpret_cast<const float4*>(&kid[i][ay][ax + 4]);
            v[i][0] = a.x; v[i][1] = a.y; v[i][2] = a.z; v[i][3] = a.w;
        }
    }
    float r[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        if (ALL4) {
            float s = v[0][c], comp = 0.0f;
            two_sum_add(s, comp, v[1][c]);
            two_sum_add(s, comp, v[2][c]);
            two_sum_add(s, comp, v[3][c]);
            r[c] = __fmul_rn(__fadd_rn(s, comp), 0.25f);
        } else {
            float s = 0.0f, comp = 0.0f;
            bool first = true;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (ci[i] < 0) continue;
                if (first) { s = v[i][c]; first = false; }
                else two_sum_add(s, comp, v[i][c]);
            }
            r[c] = div_n(__fadd_rn(s, comp), n);
        }
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

__device__ __forceinline__ float avg1(const float (*kid)[AH][KW], int ay, int ax, const int* ci, int n) {
    float s = 0.0f, comp = 0.0f;
    bool first = true;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (ci[i] < 0) continue;
        const float v = kid[i][ay][ax + ((i >= 2) ? 1 : -1) + 3];
        if (first) { s = v; first = false; }
        else two_sum_add(s, comp, v);
    }
    return div_n(__fadd_rn(s, comp), n);
}

// Level l in [1, L-1]: grid (patch, tile).
__global__ void __launch_bounds__(LEVEL_THREADS) k_level_pool_tiled(DmGeom g, int l, const unsigned char* __restrict__ vprev,
                                                                    const unsigned char* __restrict__ vcur,
                                                                    const float* __restrict__ prev, float* __restrict__ out,
                                                                    unsigned char* __restrict__ amax, float lam) {
    __shared__ __align__(16) float kid[4][AH][KW];
    __shared__ __align__(16) float avg[AH][AWP];
    __shared__ int kid_index[4];
    const int p = blockIdx.x;
    if (!vcur[p]) return;
    const int ow = g.dw[l + 1], oh = g.dh[l + 1], opitch = g.pitch(l + 1);
    const int mw = g.dw[l], mh = g.dh[l], mpitch = g.pitch(l);
    const int tiles_x = (ow + TW - 1) / TW;
    const int rx0 = (blockIdx.y % tiles_x) * TW, ry0 = (blockIdx.y / tiles_x) * TH;
    const int qx0 = 2 * rx0 - 1, qy0 = 2 * ry0 - 1;
    const int xa = 2 * rx0 - 4;                      // aligned first staged child column
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < 4) {
        int c = dm_child(g, l, p % g.Lx, p / g.Lx, tid);
        kid_index[tid] = (c >= 0 && vprev[c]) ? c : -1;
    }
    __syncthreads();
    int ci[4];
    const float* cbase[4];
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        ci[i] = kid_index[i];
        cbase[i] = ci[i] >= 0 ? prev + (long long)ci[i] * g.psize(l) : prev;
        n += ci[i] >= 0;
    }
    // stage: child i, window rows qy0 + oy_i + [0, AH), columns xa + [0, KW)
    constexpr int ROWV = KW / 4, PER_KID = AH * ROWV;
    const unsigned kid_s = (unsigned)__cvta_generic_to_shared(&kid[0][0][0]);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int oy = (i & 1) ? 1 : -1;
        for (int e = tid; e < PER_KID; e += LEVEL_THREADS) {
            const int ay = e / ROWV, v4 = e - ay * ROWV;
            const int ry = qy0 + ay + oy, x = xa + 4 * v4;
            int bytes = 0;
            const float* src = prev;
            if (ci[i] >= 0 && ry >= 0 && ry < mh && x >= 0 && x < mw) {
                bytes = min(16, 4 * (mw - x));
                src = cbase[i] + (long long)ry * mpitch + x;
            }
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                         :: "r"(kid_s + 16u * (unsigned)(i * PER_KID + e)), "l"(src), "r"(bytes) : "memory");
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // averages: compensated sum over existing children in order i = 0..3 (the
    // first existing child starts the sum: 0 + v = v exactly, so this equals
    // starting from zero), then / n; four adjacent columns per item.
    constexpr int G4 = (AW - 1) / 4;                 // 16 groups of 4 columns, then column 64
    for (int e = tid; e < AH * G4; e += LEVEL_THREADS) {
        const int ay = e / G4, ax = 4 * (e - ay * G4);
        const float4 a = (n == 4) ? avg4<true>(kid, ay, ax, ci, n) : avg4<false>(kid, ay, ax, ci, n);
        *reinterpret_cast<float4*>(&avg[ay][ax]) = a;
    }
    for (int ay = tid; ay < AH; ay += LEVEL_THREADS) avg[ay][AW - 1] = avg1(kid, ay, AW - 1, ci, n);
    __syncthreads();
    // 3x3 / 2 max-pool over in-domain averages, first strict maximum, power
    const int rx = rx0 + lane;
    if (rx >= ow) return;
    const bool interior = qx0 >= 0 && qy0 >= 0 && qx0 + AW <= mw && qy0 + AH <= mh;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int ty = warp + 8 * h;
        const int ry = ry0 + ty;
        if (ry >= oh) break;
        float best = -INFINITY;
        int code = 4;
#pragma unroll
        for (int my = -1; my <= 1; my++) {
#pragma unroll
            for (int mx = -1; mx <= 1; mx++) {
                if (!interior) {
                    int qx = 2 * rx + mx, qy = 2 * ry + my;
                    if (qx < 0 || qy < 0 || qx >= mw || qy >= mh) continue;
                }
                float a = avg[2 * ty + 1 + my][2 * lane + 1 + mx];
                if (a > best) { best = a; code = (my + 1) * 3 + (mx + 1); }
            }
        }
        long long o = ((long long)p * oh + ry) * opitch + rx;
        out[o] = dm_powf(best, lam);
        amax[o] = (unsigned char)code;
    }
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
    float a = child_mean(k, q % mw, q / mw, mw, mh, g.pitch(l));
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
            k_level_pool_tiled<<<grid, LEVEL_THREADS, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1],
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
