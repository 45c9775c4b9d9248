// Bottom-level correlation (Eq. 3-4) on the FP32 SIMT pipes, with the first
// max-pooling + subsampling (Eq. 8-9) and rectification (Eq. 11) fused into
// the epilogue.  The unpooled level-0 volume (P0 x W2 x H2 values) is never
// written to memory: only P_0(p, r) = (max_{m} C0(p, 2r+m))^lambda and its
// argmax code.
//
// Tiling.  A CTA owns 32 atomic patches (8 warps x 4) and a tile of 8 x 15
// pooled outputs, i.e. C0 at 17 rows x 32 columns of I' positions (the
// overlap of neighbouring 3x3 windows costs 32*17/(30*16) = 13% extra
// correlations).  Lane j of a warp owns C0 column j for its warp's 4 patches
// and all 17 rows: 68 accumulators, held as 34 float2 pairs (patches 0,1 and
// 2,3) so that one packed FP32x2 fma (__ffma2_rn) updates two patches: the
// instruction issue rate, not the FMA pipes, limited the scalar version.
// The image-2 descriptor halo (20 rows x 35 columns x 9 channels, one float
// each: a lane's 32-bit loads fall in distinct banks; each value is paired
// with itself in registers for the packed fmas) and the 32 patch vectors, as
// [(dx*9+c)*4+dy][patch], are staged in shared memory by asynchronous 4-byte
// copies (zero-filled outside the images).
//
// Summation order (identical to the FP32 reference): per output,
// acc = fma(a, b, acc) over dx = 0..3, then channel c = 0..8, then dy = 0..3,
// starting from 0, then acc * (1/16).  Terms outside either image are zero
// and leave acc unchanged (all operands are non-negative).  The loop order
// (dx, c) outer / dy inner lets one column of 20 halo values in registers
// feed all 4 dy offsets of all 17 rows.
//
// Epilogue: x1/16, out-of-domain positions masked to -inf, 3x3/2 max-pool
// with the first strict maximum in scan order (row-major in the window),
// i.e. (no NaN occurs) the smallest scan index among the positions equal to
// the maximum.  Each lane first reduces its own column over the three rows
// of every pooled row (maximum and the first row reaching it); the windows
// then combine three neighbouring columns (the smallest 3 * row + column
// among the columns reaching the maximum), odd lanes 2k+1 for pooled row i
// and even lanes 2k for row i+1 at once, so 30 of 32 lanes produce an output.  Maxima and
// codes are staged in shared memory, then 240 threads raise them to lambda
// and store rows of 15 consecutive outputs.
#include "dm_internal.cuh"

namespace {

constexpr int PATCHES = 32;   // per CTA
constexpr int CROWS = 17;     // C0 rows per CTA
constexpr int CCOLS = 32;     // C0 columns per CTA (one per lane)
constexpr int HROWS = CROWS + 3;
constexpr int HCOLS = CCOLS + 3;
constexpr int PW = 15;        // pooled columns per CTA
constexpr int PH = 8;         // pooled rows per CTA
constexpr int HALO_N = HROWS * HCOLS * 9;
constexpr size_t SMEM_BYTES = (size_t)HALO_N * 4 + (size_t)144 * PATCHES * 4;

// 4-byte asynchronous global -> shared copy; n = 0 writes a zero and reads nothing.
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int n) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "r"(n) : "memory");
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__global__ void __launch_bounds__(256, 2)
k_corr0_f32(DmGeom g, const float* __restrict__ d1, const float* __restrict__ d2, float lam,
            float* __restrict__ pooled0, unsigned char* __restrict__ amax0, const float* __restrict__ amat, int n0) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* halo = reinterpret_cast<float*>(smem);                          // [HROWS][HCOLS][9]
    float* a_s = reinterpret_cast<float*>(smem + (size_t)HALO_N * 4);      // [(dx*9+c)*4+dy][patch]

    const int tiles_x = (g.dw[1] + PW - 1) / PW;
    const int rx0 = (blockIdx.x % tiles_x) * PW;
    const int ry0 = (blockIdx.x / tiles_x) * PH;
    const int p_base = blockIdx.y * PATCHES;      // rows: atomic patches, or the n0 vectors of amat
    const int W2 = g.W2, H2 = g.H2;
    const int cx0 = 2 * rx0 - 1, cy0 = 2 * ry0 - 1;     // C0 tile origin (may be -1)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // image-2 halo: pixels [cx0-2, cx0+33) x [cy0-2, cy0+18), zero outside I'
    for (int pix = tid; pix < HROWS * HCOLS; pix += 256) {
        int hx = pix % HCOLS, hy = pix / HCOLS;
        int x = cx0 - 2 + hx, y = cy0 - 2 + hy;
        bool in = (x >= 0 && y >= 0 && x < W2 && y < H2);
        const float* src = in ? d2 + ((long long)y * W2 + x) * 9 : d2;
#pragma unroll
        for (int c = 0; c < 9; c++) cp_async4(halo + pix * 9 + c, src + (in ? c : 0), in ? 4 : 0);
    }
    // patch vectors: window [p-2, p+1]^2 of I, zero outside I (partial
    // patches), or row p of amat (element (dy*4 + dx)*9 + c)
    for (int k = tid; k < 144 * PATCHES; k += 256) {
        int pl = k % PATCHES, kk = k / PATCHES;
        int dy = kk % 4, c = (kk / 4) % 9, dx = kk / 36;
        int p = p_base + pl;
        const float* src = amat ? amat : d1;
        int n = 0;
        if (p < n0) {
            if (amat) {
                src = amat + (long long)p * 144 + (dy * 4 + dx) * 9 + c;
                n = 4;
            } else {
                int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
                int x = px - 2 + dx, y = py - 2 + dy;
                if (x < g.W1 && y < g.H1) {
                    src = d1 + ((long long)y * g.W1 + x) * 9 + c;
                    n = 4;
                }
            }
        }
        cp_async4(a_s + k, src, n);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();

    float2 acc01[CROWS], acc23[CROWS];
#pragma unroll
    for (int r = 0; r < CROWS; r++) {
        acc01[r] = make_float2(0.0f, 0.0f);
        acc23[r] = make_float2(0.0f, 0.0f);
    }

    const float4* a4p = reinterpret_cast<const float4*>(a_s) + warp;   // 4 patches of this warp
#pragma unroll 1
    for (int dx = 0; dx < 4; dx++) {
#pragma unroll 1
        for (int c = 0; c < 9; c++) {
            float h[HROWS];
#pragma unroll
            for (int r = 0; r < HROWS; r++) h[r] = halo[(r * HCOLS + lane + dx) * 9 + c];
#pragma unroll
            for (int dy = 0; dy < 4; dy++) {
                float4 a = a4p[((dx * 9 + c) * 4 + dy) * (PATCHES / 4)];
                float2 a01 = make_float2(a.x, a.y), a23 = make_float2(a.z, a.w);
#pragma unroll
                for (int r = 0; r < CROWS; r++) {
                    const float2 hh = make_float2(h[r + dy], h[r + dy]);
                    acc01[r] = __ffma2_rn(a01, hh, acc01[r]);
                    acc23[r] = __ffma2_rn(a23, hh, acc23[r]);
                }
            }
        }
    }
    __syncthreads();   // halo and patch vectors are no longer needed: reuse the space

    float* best_s = reinterpret_cast<float*>(smem);                                  // [32][PH][PW]
    unsigned char* code_s = smem + (size_t)PATCHES * PH * PW * 4;                    // [32][PH][PW]
    const int cx = cx0 + lane;
    const bool col_in = (cx >= 0 && cx < W2);
    const bool odd = lane & 1;
    const bool writer = lane < 2 * PW;             // lane 2k+1: column k of row i; lane 2k: column k of row i+1
    const int row_sh = odd ? 0 : 4;                // this lane's pooled row (i or i+1) in a packed pair
#pragma unroll
    for (int q = 0; q < 4; q++) {
        float v[CROWS];
#pragma unroll
        for (int r = 0; r < CROWS; r++) {
            float a = (q == 0) ? acc01[r].x : (q == 1) ? acc01[r].y : (q == 2) ? acc23[r].x : acc23[r].y;
            int cy = cy0 + r;
            v[r] = (col_in && cy >= 0 && cy < H2) ? __fmul_rn(a, 0.0625f) : -INFINITY;
        }
        // this column's maximum over the rows 2i..2i+2 of each pooled row i,
        // and 3 x its first row reaching it, packed 4 bits per pooled row
        float cm[PH];
        uint32_t cyp = 0;
#pragma unroll
        for (int i = 0; i < PH; i++) {
            cm[i] = fmax3(v[2 * i], v[2 * i + 1], v[2 * i + 2]);
            const uint32_t y3 = v[2 * i] == cm[i] ? 0u : (v[2 * i + 1] == cm[i] ? 3u : 6u);
            cyp |= y3 << (4 * i);
        }
        // the neighbours' columns: x0 | x1 | x2 of the window this lane pools
        const uint32_t cyx = __shfl_xor_sync(0xffffffffu, cyp, 1);
        const uint32_t cy1 = __shfl_down_sync(0xffffffffu, cyp, 1);
        const uint32_t cy2 = __shfl_down_sync(0xffffffffu, cyp, 2);
        const uint32_t y0p = odd ? cyx : cyp, y1p = odd ? cyp : cyx, y2p = odd ? cy1 : cy2;
        const int pl = warp * 4 + q;
#pragma unroll
        for (int i = 0; i < PH; i += 2) {
            const float r = __shfl_xor_sync(0xffffffffu, odd ? cm[i + 1] : cm[i], 1);
            const float d1v = __shfl_down_sync(0xffffffffu, cm[i], 1);
            const float d2v = __shfl_down_sync(0xffffffffu, cm[i + 1], 2);
            const float x0 = odd ? r : cm[i + 1];
            const float x1 = odd ? cm[i] : r;
            const float x2 = odd ? d1v : d2v;
            const float best = fmax3(x0, x1, x2);
            const int sh = 4 * i + row_sh;
            const int k0 = x0 == best ? (int)((y0p >> sh) & 15u) : 15;
            const int k1 = x1 == best ? (int)((y1p >> sh) & 15u) + 1 : 15;
            const int k2 = x2 == best ? (int)((y2p >> sh) & 15u) + 2 : 15;
            const int code = min(k0, min(k1, k2));
            if (writer) {
                const int e = (pl * PH + i + (odd ? 0 : 1)) * PW + (lane >> 1);
                best_s[e] = best;
                code_s[e] = (unsigned char)code;
            }
        }
    }
    __syncthreads();
    // 240 threads raise the staged maxima to lambda: thread t keeps column
    // t % 15 and pooled row (t / 15) % 8, and takes every second patch from
    // t / 120, two patches per packed evaluation (bit-identical to dm_powf
    // lane by lane); consecutive threads store consecutive outputs of a row
    if (tid < 16 * PW) {
        const int kk = tid % PW, u0 = tid / PW;
        const int rx = rx0 + kk, ry = ry0 + (u0 % PH);
        const int mw = g.dw[1], mh = g.dh[1];
        if (rx < mw && ry < mh) {
            const int pl0 = u0 / PH;
            const long long pstride = (long long)mh * g.pitch(1);
            const long long o0 = ((long long)(p_base + pl0) * mh + ry) * g.pitch(1) + rx;
#pragma unroll 2
            for (int j = 0; j < PATCHES / 2; j += 2) {
                const int e = tid + j * 16 * PW;
                const float2 v = dm_powf2(make_float2(best_s[e], best_s[e + 16 * PW]), lam);
                const int p = p_base + pl0 + 2 * j;
                const long long o = o0 + 2 * j * pstride;
                if (p < n0) {
                    pooled0[o] = v.x;
                    amax0[o] = code_s[e];
                }
                if (p + 2 < n0) {
                    pooled0[o + 2 * pstride] = v.y;
                    amax0[o + 2 * pstride] = code_s[e + 16 * PW];
                }
            }
        }
    }
}

}  // namespace

cudaError_t dm_launch_corr0_f32(const DmGeom& g, const float* d1, const float* d2, float lam, float* pooled0,
                                unsigned char* amax0, cudaStream_t st, const float* amat, int n_rows) {
    if (n_rows < 0) n_rows = g.P0x * g.P0y;
    int tiles = ((g.dw[1] + PW - 1) / PW) * ((g.dh[1] + PH - 1) / PH);
    int pblocks = (n_rows + PATCHES - 1) / PATCHES;
    dim3 grid(tiles, pblocks);
    static std::atomic<unsigned long long> smem_done{0};   // > 48 KB dynamic shared memory opted in, per device
    cudaError_t e = dm_smem_opt_in(reinterpret_cast<const void*>(k_corr0_f32), (int)SMEM_BYTES, smem_done);
    if (e != cudaSuccess) return e;
    k_corr0_f32<<<grid, 256, SMEM_BYTES, st>>>(g, d1, d2, lam, pooled0, amax0, amat, n_rows);
    dm_count_launches(1);
    return cudaGetLastError();
}
