// Pyramid levels l >= 1 (Eq. 5-12, boundary rule of Sec. 3.2, Algorithm 1).
//
// For a lattice patch p at level l with existing children c_i = p + 2^l o_i:
//   C_l(p, q) = (1/n) sum_{existing i} P_{l-1}(c_i, q + o_i)      (0 outside the domain)
// and, below the top, the stored pooled map
//   P_l(p, r) = (max over in-domain m of C_l(p, 2r + m))^lambda   + argmax code,
// or at the top C_L(p, q) = (C_l(p, q))^lambda.
// The children's sum runs in child order i = 0..3, Knuth-TwoSum compensated
// and rounded once (default) or plain (one rounding per addition), then is
// divided by n; pooling is on the unrectified average and the power is
// applied to the pooled value (x -> x^lambda is increasing on [0,1]).
//
// This pass streams the pooled maps of the level below (bandwidth) and does
// a fixed amount of arithmetic per stored output (~4 averages of 4 values,
// a 9-way max with argmax, one power): it is bound by instruction issue.  A CTA owns one patch and a tile of
// 32 x 16 pooled outputs (two per thread): one thread stages the 4 child-map
// windows it needs (72 x 33 floats each) in shared memory with 3-D TMA tensor
// loads (rows of the pooled maps are padded to 16 floats and the window's
// first column is a multiple of 4, so every load starts 16-byte aligned; the
// tensor map zero-fills whatever lies outside the domain), the CTA forms the
// 65 x 33 averages once, then pools them.  Patches vary fastest in the grid,
// so the (up to 4) parents that read the same child window run at about the
// same time and the repeat reads hit L2.  Algorithmic bytes per stored
// output: 16 B of child values read (each child value is shared by 4
// parents), 4 + 1 B written.
#include "dm_internal.cuh"

namespace {

// valid[l][p] = 1 iff some child exists (Eq. 7 with the boundary rule), and
// kids[p] = the existing children (index into level l-1, -1 where absent).
__global__ void k_valid(DmGeom g, int l, const unsigned char* __restrict__ vprev, unsigned char* __restrict__ v,
                        int4* __restrict__ kids) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.Lx * g.Ly) return;
    int ix = p % g.Lx, iy = p / g.Lx;
    int c[4];
    unsigned char any = 0;
    for (int i = 0; i < 4; i++) {
        c[i] = dm_child(g, l, ix, iy, i);
        if (c[i] >= 0 && !vprev[c[i]]) c[i] = -1;
        if (c[i] >= 0) any = 1;
    }
    v[p] = any;
    kids[p] = make_int4(c[0], c[1], c[2], c[3]);
}

__global__ void k_fill_u8(unsigned char* p, int n, unsigned char val) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = val;
}

struct Kids {
    const float* base[4];
    int n;
};

// Knuth TwoSum step of the compensated child sum.
__device__ __forceinline__ void two_sum_add(float& s, float& comp, float v) {
    const float t = __fadd_rn(s, v);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    s = t;
    comp = __fadd_rn(comp, err);
}

// Child sum step: compensated or plain.  The first existing child starts the
// sum (0 + v = v exactly, the same as starting from zero).
template <bool COMP>
__device__ __forceinline__ void child_add(float& s, float& comp, float v) {
    if (COMP) two_sum_add(s, comp, v);
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

constexpr int TW = 32;                           // pooled columns per CTA tile (one per lane)
constexpr int AW = 2 * TW + 1;                   // average columns per CTA (65)
constexpr int KW = 72;                           // staged child columns (TMA box width)
constexpr int AWP = 68;                          // padded row of the averages (16-byte aligned rows)
constexpr int LEVEL_THREADS = 256;

// CTA tile of TW x TH pooled outputs (TH = 8 or 16, chosen by the autotuner):
// AH rows of averages, child windows of KW x AH floats (KIDF with padding to
// 128 bytes), KID_BYTES delivered by one TMA window load.
template <int TH_>
struct LevelTile {
    static constexpr int TH = TH_;
    static constexpr int AH = 2 * TH + 1;
    static constexpr int KIDF = ((AH * KW + 31) / 32) * 32;
    static constexpr unsigned KID_BYTES = AH * KW * 4;
};
constexpr long long LEVEL_WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

// x / n rounded once, for n in 1..4: multiplications by 1, 1/2, 1/4 are exact,
// so they equal the correctly rounded quotient; n = 3 divides.
__device__ __forceinline__ float div_n(float x, int n) {
    return n == 3 ? __fdiv_rn(x, 3.0f) : __fmul_rn(x, n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.0f));
}

// Averages at staged row ay, columns ax .. ax+3 of child 0's frame, from the
// four child windows: child i contributes kid[i][ay][ax + ox_i + 3].
template <int KIDF, bool COMP, bool ALL4>
__device__ __forceinline__ float4 avg4(const float* kid, int ay, int ax, const int* ci, int n) {
    // children with ox = -1 (i = 0, 1) read columns ax+2 .. ax+5 (8-byte aligned),
    // children with ox = +1 (i = 2, 3) read columns ax+4 .. ax+7 (16-byte aligned)
    float v[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (!ALL4 && ci[i] < 0) continue;
        const float* row = kid + i * KIDF + ay * KW;
        if (i < 2) {
            const float2 a = *reinterpret_cast<const float2*>(row + ax + 2);
            const float2 b = *reinterpret_cast<const float2*>(row + ax + 4);
            v[i][0] = a.x; v[i][1] = a.y; v[i][2] = b.x; v[i][3] = b.y;
        } else {
            const float4 a = *reinterpret_cast<const float4*>(row + ax + 4);
            v[i][0] = a.x; v[i][1] = a.y; v[i][2] = a.z; v[i][3] = a.w;
        }
    }
    float r[4];
#pragma unroll
    for (int c = 0; c < 4; c++) {
        float s = 0.0f, comp = 0.0f;
        if (ALL4) {
            s = v[0][c];
            child_add<COMP>(s, comp, v[1][c]);
            child_add<COMP>(s, comp, v[2][c]);
            child_add<COMP>(s, comp, v[3][c]);
            r[c] = __fmul_rn(COMP ? __fadd_rn(s, comp) : s, 0.25f);
        } else {
#pragma unroll
            for (int i = 0; i < 4; i++)
                if (ci[i] >= 0) child_add<COMP>(s, comp, v[i][c]);
            r[c] = div_n(COMP ? __fadd_rn(s, comp) : s, n);
        }
    }
    return make_float4(r[0], r[1], r[2], r[3]);
}

template <int KIDF, bool COMP>
__device__ __forceinline__ float avg1(const float* kid, int ay, int ax, const int* ci, int n) {
    float s = 0.0f, comp = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        if (ci[i] < 0) continue;
        child_add<COMP>(s, comp, kid[i * KIDF + ay * KW + ax + ((i >= 2) ? 1 : -1) + 3]);
    }
    return div_n(COMP ? __fadd_rn(s, comp) : s, n);
}

// Level l in [1, L-1]: grid (patch, tile).  `tmap` maps the pooled maps of
// level l-1 as a 3-D array (columns dw[l], rows dh[l], patches) with a
// 72 x 33 x 1 box.
template <bool COMP, int TH>
__global__ void __launch_bounds__(LEVEL_THREADS) k_level_pool_tiled(DmGeom g, int l, const __grid_constant__ CUtensorMap tmap,
                                                                    const int4* __restrict__ kids,
                                                                    float* __restrict__ out,
                                                                    unsigned char* __restrict__ amax, float lam,
                                                                    int* __restrict__ err) {
    using T = LevelTile<TH>;
    constexpr int AH = T::AH, KIDF = T::KIDF;
    __shared__ __align__(128) float kid[4 * KIDF];
    __shared__ __align__(16) float avg[AH][AWP];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_s;
    const int p = blockIdx.x;
    // the patch's existing children (one broadcast load); none: the patch does not exist
    const int4 kc = __ldg(kids + p);
    const int ci[4] = {kc.x, kc.y, kc.z, kc.w};
    const int n = (ci[0] >= 0) + (ci[1] >= 0) + (ci[2] >= 0) + (ci[3] >= 0);
    if (n == 0) return;
    const int ow = g.dw[l + 1], oh = g.dh[l + 1], opitch = g.pitch(l + 1);
    const int mw = g.dw[l], mh = g.dh[l];
    const int tiles_x = (ow + TW - 1) / TW;
    const int rx0 = (blockIdx.y % tiles_x) * TW, ry0 = (blockIdx.y / tiles_x) * TH;
    const int qx0 = 2 * rx0 - 1, qy0 = 2 * ry0 - 1;
    const int xa = 2 * rx0 - 4;                      // first staged child column (multiple of 4: 16-byte aligned)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t bar_s = (uint32_t)__cvta_generic_to_shared(&bar);
    // stage: child i, window rows qy0 + oy_i + [0, AH), columns xa + [0, KW)
    if (tid == 0) {
        abort_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bar_s) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar_s), "r"(T::KID_BYTES * n) : "memory");
        const uint32_t kid_s = (uint32_t)__cvta_generic_to_shared(kid);
#pragma unroll
        for (int i = 0; i < 4; i++) {
            if (ci[i] < 0) continue;
            const int oy = (i & 1) ? 1 : -1;
            asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                         :: "r"(kid_s + (uint32_t)(i * KIDF * 4)), "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(xa),
                            "r"(qy0 + oy), "r"(ci[i]), "r"(bar_s)
                         : "memory");
        }
    }
    __syncthreads();                                 // barrier initialised
    {
        const long long t0 = clock64();
        uint32_t done = 0;
        while (!done) {
            asm volatile("{.reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0; selp.u32 %0, 1, 0, q;}"
                         : "=r"(done) : "r"(bar_s) : "memory");
            if (!done && clock64() - t0 > LEVEL_WAIT_CYCLES) {
                atomicOr(err, 1);
                abort_s = 1;
                break;
            }
        }
    }
    __syncthreads();
    if (abort_s) return;
    // averages: sum over existing children in order i = 0..3, then / n; four
    // adjacent columns per item.
    constexpr int G4 = (AW - 1) / 4;                 // 16 groups of 4 columns, then column 64
    for (int e = tid; e < AH * G4; e += LEVEL_THREADS) {
        const int ay = e / G4, ax = 4 * (e - ay * G4);
        const float4 a = (n == 4) ? avg4<KIDF, COMP, true>(kid, ay, ax, ci, n) : avg4<KIDF, COMP, false>(kid, ay, ax, ci, n);
        *reinterpret_cast<float4*>(&avg[ay][ax]) = a;
    }
    for (int ay = tid; ay < AH; ay += LEVEL_THREADS) avg[ay][AW - 1] = avg1<KIDF, COMP>(kid, ay, AW - 1, ci, n);
    __syncthreads();
    // 3x3 / 2 max-pool over in-domain averages, first strict maximum, power.
    // A thread owns R = TH/8 vertically adjacent outputs (rows R*warp ..), so
    // the horizontal 3-maxima of the 2R+1 average rows it reads are formed once
    // (a row shared by two outputs serves both); rows are then merged in scan
    // order m_y = -1, 0, 1, which keeps the first strict maximum.
    constexpr int R = TH / 8;
    const int rx = rx0 + lane;
    if (rx >= ow) return;
    const bool interior = qx0 >= 0 && qy0 >= 0 && qx0 + AW <= mw && qy0 + AH <= mh;
    const int ty0 = R * warp;
    float hv[2 * R + 1];
    int hc[2 * R + 1];
#pragma unroll
    for (int k = 0; k < 2 * R + 1; k++) {
        const int ay = 2 * ty0 + k;                  // average row; map row qy0 + ay
        const int qy = qy0 + ay;
        float best = -INFINITY;
        int code = 0;
        if (interior || (qy >= 0 && qy < mh)) {
#pragma unroll
            for (int mx = -1; mx <= 1; mx++) {
                if (!interior) {
                    const int qx = 2 * rx + mx;
                    if (qx < 0 || qx >= mw) continue;
                }
                const float a = avg[ay][2 * lane + 1 + mx];
                if (a > best) { best = a; code = mx + 1; }
            }
        }
        hv[k] = best;
        hc[k] = code;
    }
#pragma unroll
    for (int j = 0; j < R; j++) {
        const int ry = ry0 + ty0 + j;
        if (ry >= oh) break;
        float best = -INFINITY;
        int code = 4;
#pragma unroll
        for (int my = 0; my < 3; my++) {
            const float v = hv[2 * j + my];
            if (v > best) { best = v; code = my * 3 + hc[2 * j + my]; }
        }
        long long o = ((long long)p * oh + ry) * opitch + rx;
        out[o] = dm_powf(best, lam);
        amax[o] = (unsigned char)code;
    }
}

// Top level L: C_L = (mean of children)^lambda over the domain of level L.
template <bool COMP>
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
    float a = child_mean<COMP>(k, q % mw, q / mw, mw, mh, g.pitch(l));
    top[(long long)p * mw * mh + q] = dm_powf(a, lam);
}

}  // namespace

cudaError_t dm_launch_levels(const DmGeom& g, const dm_pyramid& py, float lam, int* status, cudaStream_t st) {
    const int B = 128;
    int n0 = g.npatch(0), np = g.npatch(1);
    k_fill_u8<<<(n0 + 255) / 256, 256, 0, st>>>(const_cast<unsigned char*>(py.valid[0]), n0, 1);
    for (int l = 1; l <= g.L; l++) {
        k_valid<<<(np + 255) / 256, 256, 0, st>>>(g, l, py.valid[l - 1], const_cast<unsigned char*>(py.valid[l]), py.kids);
        if (l < g.L) {
            // pooled maps of level l-1: [npatch(l-1)][dh[l]][pitch(l)] floats
            const int th = py.tune.level_th == 8 ? 8 : 16;
            CUtensorMap tm;
            const cuuint64_t dims[3] = {(cuuint64_t)g.dw[l], (cuuint64_t)g.dh[l], (cuuint64_t)g.npatch(l - 1)};
            const cuuint64_t strides[2] = {(cuuint64_t)g.pitch(l) * 4, (cuuint64_t)g.psize(l) * 4};
            const cuuint32_t box[3] = {KW, (cuuint32_t)(2 * th + 1), 1};
            if (!dm_encode_tiled(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(py.pooled[l - 1]), dims,
                                 strides, box))
                return cudaErrorNotSupported;
            int tiles = ((g.dw[l + 1] + TW - 1) / TW) * ((g.dh[l + 1] + th - 1) / th);
            dim3 grid(np, tiles);
            auto kern = th == 8 ? (py.compensated ? k_level_pool_tiled<true, 8> : k_level_pool_tiled<false, 8>)
                                : (py.compensated ? k_level_pool_tiled<true, 16> : k_level_pool_tiled<false, 16>);
            kern<<<grid, LEVEL_THREADS, 0, st>>>(g, l, tm, py.kids, const_cast<float*>(py.pooled[l]),
                                                 const_cast<unsigned char*>(py.amax[l]), lam, status);
        } else {
            int n = g.dw[l] * g.dh[l];
            dim3 grid((n + B - 1) / B, np);
            auto kern = py.compensated ? k_level_top<true> : k_level_top<false>;
            kern<<<grid, B, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1], const_cast<float*>(py.top), lam);
        }
    }
    dm_count_launches(1 + 2 * g.L);
    return cudaGetLastError();
}
