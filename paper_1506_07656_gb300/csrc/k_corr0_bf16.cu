// Bottom-level correlation (Eq. 3-4) on the 5th-generation tensor cores:
// tcgen05.mma kind::f16 with BF16 operands and FP32 accumulation in tensor
// memory, with the first max-pooling + subsampling (Eq. 8-9) and the
// rectification (Eq. 11) fused into the epilogue.  The unpooled level-0
// volume never reaches global memory.
//
// GEMM view.  D[m][n] = sum_k A[m][k] B[n][k], m an atomic patch of I,
// n a position of I', k = (dy*4 + dx)*9 + c over the 4x4x9 window (K = 144,
// nine MMAs of K = 16).  C0 = D / 16.
//   A: the patch vectors, packed once per call by k_pack_a into 128-row tiles
//      in the no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core
//      matrix; 18 core matrices along K per 8-row group, 2304 bytes), so one
//      36,864-byte bulk copy (cp.async.bulk, TMA engine) moves a tile to
//      shared memory.
//   B: the implicit im2col of I' for one N-tile of 17 x 15 positions (255 of
//      the 256 rows), built in shared memory by all warps in the same layout
//      and kept resident while the CTA sweeps a chunk of up to 110 M-tiles.
//   D: 128 lanes x 256 FP32 columns of TMEM; two accumulators (512 columns)
//      let the epilogue drain one tile while the next is multiplied.
// Pooling geometry: the N-tile's positions are x = 2 rx0 - 1 + lx (lx < 17),
// y = 2 ry0 - 1 + ly (ly < 15); they cover the 3x3 windows of the 8 x 7
// pooled outputs (rx0 + k, ry0 + j), centre lx = 2k + 1, ly = 2j + 1.
//
// Warp roles (448 threads, one CTA per SM, persistent over work units
// (N-tile, M-chunk)): warp 0 issues the bulk copies of A (3-stage ring),
// warp 1 allocates TMEM and one lane issues the MMAs and commits, warps 2-13
// drain the accumulators: three warps per TMEM lane quadrant, each on a band
// of pooled rows (0-2, 3-4, 5-6), read them with tcgen05.ld, pool with the
// first-strict-maximum argmax rule (scan my = -1..1, then mx), and store
// P_0 = (max / 16)^lambda (MUFU-based power) and the argmax code.  Twelve
// draining warps keep enough independent work in flight to hide ALU latency;
// four were latency-bound.
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// *err, stops issuing work, releases TMEM and returns.
#include <cuda_bf16.h>

#include "dm_internal.cuh"

namespace {

constexpr int BM = 128;                       // patches per M-tile (TMEM lanes)
constexpr int KD = 144;                       // 4 x 4 x 9
constexpr int KSTEPS = KD / 16;               // MMAs per tile
constexpr int CX = 17, CY = 15;               // C0 positions per N-tile
constexpr int BN = 256;                       // CX * CY = 255, padded
constexpr int PX = 8, PY = 7;                 // pooled outputs per N-tile
constexpr int GROUP = (KD / 8) * 128;         // 2304 bytes per 8-row group
constexpr int A_TILE = BM * KD * 2;           // 36864
constexpr int B_TILE = BN * KD * 2;           // 73728
constexpr int STAGES = 3;
constexpr int M_CHUNK = 110;                  // M-tiles per work unit
constexpr int EPI_WARPS = 12;
constexpr int THREADS = 64 + 32 * EPI_WARPS;
constexpr size_t SMEM = (size_t)B_TILE + (size_t)STAGES * A_TILE + 256;
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address,
// leading-dimension byte offset (between core matrices along K), stride byte
// offset (between 8-row groups), fixed field 0b001 at bit 46.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((uint32_t)(GROUP >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor kind::f16: D = F32, A = B = BF16, both K-major, N, M
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
    long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p;}"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
        if (*abort_flag) return false;
        if (clock64() - t0 > WAIT_CYCLES) {
            atomicOr(err, 1);
            *abort_flag = 1;
            return false;
        }
    }
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

// Pack the patch vectors of I into BF16 M-tiles (zero rows past the last patch).
__global__ void k_pack_a(DmGeom g, const float* __restrict__ d1, __nv_bfloat16* __restrict__ a16, int n_mtiles) {
    const long long total = (long long)n_mtiles * BM * (KD / 8);
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int kc = (int)(idx % (KD / 8));
    const int pm = (int)(idx / (KD / 8));
    const int n0 = g.P0x * g.P0y;
    __align__(16) __nv_bfloat16 v[8];
    const int px = 4 * (pm % g.P0x) + 2, py = 4 * (pm / g.P0x) + 2;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        int k = kc * 8 + e;
        int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
        int x = px - 2 + dx, y = py - 2 + dy;
        float f = (pm < n0 && x < g.W1 && y < g.H1) ? __ldg(d1 + ((long long)y * g.W1 + x) * 9 + c) : 0.0f;
        v[e] = __float2bfloat16_rn(f);
    }
    const int t = pm / BM, r = pm % BM;
    char* dst = reinterpret_cast<char*>(a16) + (long long)t * A_TILE + (r >> 3) * GROUP + kc * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
}

struct EpiArgs {
    uint32_t taddr;     // TMEM address of this warp's lane quadrant, column 0
    int row;            // accumulator row (patch within the M-tile)
    int m0, cx0, cy0, rx0, ry0, W2, H2, mw, mh, pitch, n0;
    float lam;
    bool interior;      // every C0 position of the N-tile lies inside I'
};

// Pool pooled rows [J0, J1) of one accumulator (C0 rows 2*J0 .. 2*J1) for this
// thread's patch, release the accumulator, then store.
template <int J0, int J1>
__device__ __forceinline__ void epilogue_band(const EpiArgs& e, uint32_t b, int j, uint32_t bar_empty,
                                              float* __restrict__ pooled0, unsigned char* __restrict__ amax0) {
    constexpr int NJ = J1 - J0;
    float best[NJ][PX];
    int code[NJ][PX];
#pragma unroll
    for (int y = 0; y < NJ; y++)
#pragma unroll
        for (int x = 0; x < PX; x++) { best[y][x] = -INFINITY; code[y][x] = 4; }
    const uint32_t taddr = e.taddr + b * BN;
#pragma unroll
    for (int ly = 2 * J0; ly <= 2 * J1; ly++) {
        uint32_t r[CX];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                     : "r"(taddr + ly * CX));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[16]) : "r"(taddr + ly * CX + 16));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float v[CX];
#pragma unroll
        for (int lx = 0; lx < CX; lx++) v[lx] = __uint_as_float(r[lx]);
        if (!e.interior) {
            const int ty = e.cy0 + ly;
            const bool rin = ty >= 0 && ty < e.H2;
#pragma unroll
            for (int lx = 0; lx < CX; lx++) {
                const int tx = e.cx0 + lx;
                if (!(rin && tx >= 0 && tx < e.W2)) v[lx] = -INFINITY;
            }
        }
#pragma unroll
        for (int k = 0; k < PX; k++) {
            float h = v[2 * k];
            int hc = 0;
            if (v[2 * k + 1] > h) { h = v[2 * k + 1]; hc = 1; }
            if (v[2 * k + 2] > h) { h = v[2 * k + 2]; hc = 2; }
            // C0 row ly is m_y = -1 of pooled row ly/2 (even ly), m_y = 0 of (ly-1)/2 (odd),
            // m_y = +1 of ly/2 - 1 (even ly); rows arrive in scan order
            if ((ly & 1) == 0) {
                if (ly / 2 - 1 >= J0) {
                    const int jj = ly / 2 - 1 - J0;
                    if (h > best[jj][k]) { best[jj][k] = h; code[jj][k] = 6 + hc; }
                }
                if (ly / 2 < J1) {
                    const int jj = ly / 2 - J0;
                    if (h > best[jj][k]) { best[jj][k] = h; code[jj][k] = hc; }
                }
            } else {
                const int jj = (ly - 1) / 2 - J0;
                if (h > best[jj][k]) { best[jj][k] = h; code[jj][k] = 3 + hc; }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(bar_empty);
    const int p = (e.m0 + j) * BM + e.row;
    if (p >= e.n0) return;
#pragma unroll
    for (int y = 0; y < NJ; y++) {
        const int ry = e.ry0 + J0 + y;
        if (ry >= e.mh) break;
        // rows are padded to a multiple of 8 floats and rx0 is a multiple of 8, so the
        // 8 outputs of a row always fit and are 32-byte aligned (padding columns
        // receive values that nothing reads)
        const long long o = ((long long)p * e.mh + ry) * e.pitch + e.rx0;
        {
            float4 f0, f1;
            f0.x = __powf(best[y][0] * 0.0625f, e.lam); f0.y = __powf(best[y][1] * 0.0625f, e.lam);
            f0.z = __powf(best[y][2] * 0.0625f, e.lam); f0.w = __powf(best[y][3] * 0.0625f, e.lam);
            f1.x = __powf(best[y][4] * 0.0625f, e.lam); f1.y = __powf(best[y][5] * 0.0625f, e.lam);
            f1.z = __powf(best[y][6] * 0.0625f, e.lam); f1.w = __powf(best[y][7] * 0.0625f, e.lam);
            *reinterpret_cast<float4*>(pooled0 + o) = f0;
            *reinterpret_cast<float4*>(pooled0 + o + 4) = f1;
            uint2 cc;
            cc.x = (uint32_t)code[y][0] | ((uint32_t)code[y][1] << 8) | ((uint32_t)code[y][2] << 16) | ((uint32_t)code[y][3] << 24);
            cc.y = (uint32_t)code[y][4] | ((uint32_t)code[y][5] << 8) | ((uint32_t)code[y][6] << 16) | ((uint32_t)code[y][7] << 24);
            *reinterpret_cast<uint2*>(amax0 + o) = cc;
        }
    }
}

__global__ void __launch_bounds__(THREADS, 1)
k_corr0_tc(DmGeom g, const __nv_bfloat16* __restrict__ a16, const float* __restrict__ d2, float lam,
           float* __restrict__ pooled0, unsigned char* __restrict__ amax0, int n_mtiles, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem;
    unsigned char* sA = smem + B_TILE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sA + STAGES * A_TILE);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + STAGES);
    const uint32_t bar_acc_full = smem_u32(bars + 2 * STAGES), bar_acc_empty = smem_u32(bars + 2 * STAGES + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(bar_acc_full + 8 * b, 1);
            mbar_init(bar_acc_empty + 8 * b, 32 * EPI_WARPS);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tmem_holder)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_holder;

    const int W2 = g.W2, H2 = g.H2, mw = g.dw[1], mh = g.dh[1], pitch = g.pitch(1);
    const int n0 = g.P0x * g.P0y;
    const int tiles_x = (mw + PX - 1) / PX, tiles_y = (mh + PY - 1) / PY;
    const int mchunks = (n_mtiles + M_CHUNK - 1) / M_CHUNK;
    const int n_units = tiles_x * tiles_y * mchunks;
    uint32_t a_it = 0, acc_it = 0;

    for (int unit = blockIdx.x; unit < n_units; unit += gridDim.x) {
        const int ntile = unit / mchunks, mc = unit % mchunks;
        const int m0 = mc * M_CHUNK, m1 = min(n_mtiles, m0 + M_CHUNK), nt = m1 - m0;
        const int rx0 = (ntile % tiles_x) * PX, ry0 = (ntile / tiles_x) * PY;
        const int cx0 = 2 * rx0 - 1, cy0 = 2 * ry0 - 1;

        // B: implicit im2col of I' for this N-tile (zero outside I' and in row 255)
        for (int ch = tid; ch < BN * (KD / 8); ch += THREADS) {
            const int n = ch / (KD / 8), kc = ch % (KD / 8);
            const int lx = n % CX, ly = n / CX;
            const int tx = cx0 + lx, ty = cy0 + ly;
            __align__(16) __nv_bfloat16 v[8];
#pragma unroll
            for (int e = 0; e < 8; e++) {
                int k = kc * 8 + e;
                int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
                int x = tx - 2 + dx, y = ty - 2 + dy;
                float f = (n < CX * CY && x >= 0 && y >= 0 && x < W2 && y < H2) ? __ldg(d2 + ((long long)y * W2 + x) * 9 + c) : 0.0f;
                v[e] = __float2bfloat16_rn(f);
            }
            *reinterpret_cast<uint4*>(sB + (n >> 3) * GROUP + kc * 128 + (n & 7) * 16) = *reinterpret_cast<const uint4*>(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                for (int j = 0; j < nt; j++) {
                    const uint32_t it = a_it + j, s = it % STAGES, ph = (it / STAGES) & 1;
                    if (!mbar_wait(bar_empty + 8 * s, ph ^ 1, abort_flag, err)) break;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar_full + 8 * s), "r"(A_TILE) : "memory");
                    const char* src = reinterpret_cast<const char*>(a16) + (long long)(m0 + j) * A_TILE;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(smem_u32(sA + s * A_TILE)), "l"(src), "r"(A_TILE), "r"(bar_full + 8 * s) : "memory");
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                for (int j = 0; j < nt; j++) {
                    const uint32_t it = a_it + j, s = it % STAGES, ph = (it / STAGES) & 1;
                    const uint32_t ai = acc_it + j, b = ai & 1, aph = (ai >> 1) & 1;
                    if (!mbar_wait(bar_full + 8 * s, ph, abort_flag, err)) break;
                    if (!mbar_wait(bar_acc_empty + 8 * b, aph ^ 1, abort_flag, err)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d_tmem = tmem + b * BN;
                    const uint32_t a_base = smem_u32(sA + s * A_TILE), b_base = smem_u32(sB);
#pragma unroll
                    for (int k = 0; k < KSTEPS; k++) {
                        uint64_t ad = make_desc(a_base + k * 256), bd = make_desc(b_base + k * 256);
                        uint32_t acc = k > 0;
                        asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}"
                                     :: "r"(d_tmem), "l"(ad), "l"(bd), "r"(IDESC), "r"(acc) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar_empty + 8 * s) : "memory");
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar_acc_full + 8 * b) : "memory");
                }
            }
        } else {
            // epilogue: warp w drains TMEM lane quadrant w % 4, pooled-row band (w - 2) / 4
            const int quad = warp & 3;
            const int part = (warp - 2) >> 2;
            const bool interior = cx0 >= 0 && cy0 >= 0 && cx0 + CX <= W2 && cy0 + CY <= H2;
            const EpiArgs ea{tmem + ((uint32_t)(quad * 32) << 16), quad * 32 + lane, m0, cx0, cy0, rx0, ry0, W2, H2, mw,
                             mh, pitch, n0, lam, interior};
            for (int j = 0; j < nt; j++) {
                const uint32_t ai = acc_it + j, b = ai & 1, aph = (ai >> 1) & 1;
                if (!mbar_wait(bar_acc_full + 8 * b, aph, abort_flag, err)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (part == 0) epilogue_band<0, 3>(ea, b, j, bar_acc_empty + 8 * b, pooled0, amax0);
                else if (part == 1) epilogue_band<3, 5>(ea, b, j, bar_acc_empty + 8 * b, pooled0, amax0);
                else epilogue_band<5, 7>(ea, b, j, bar_acc_empty + 8 * b, pooled0, amax0);
            }
        }
        a_it += nt;
        acc_it += nt;
        __syncthreads();   // the epilogue has consumed every accumulator: the tensor core is done with sB
        if (*abort_flag) break;
    }
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

}  // namespace

size_t dm_corr0_bf16_a_bytes(const DmGeom& g) {
    size_t n_mtiles = ((size_t)g.npatch(0) + BM - 1) / BM;
    return n_mtiles * A_TILE;
}

cudaError_t dm_launch_corr0_bf16(const DmGeom& g, const float* d1, const float* d2, float lam, void* a16, void* status,
                                 float* pooled0, unsigned char* amax0, cudaStream_t st) {
    const int n0 = g.npatch(0);
    const int n_mtiles = (n0 + BM - 1) / BM;
    {
        long long total = (long long)n_mtiles * BM * (KD / 8);
        k_pack_a<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, d1, reinterpret_cast<__nv_bfloat16*>(a16), n_mtiles);
    }
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    static unsigned long long attr_set = 0;
    if (dev < 64 && !(attr_set & (1ull << dev))) {
        cudaError_t e = cudaFuncSetAttribute(k_corr0_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
        if (e != cudaSuccess) return e;
        attr_set |= 1ull << dev;
    }
    const int tiles = ((g.dw[1] + PX - 1) / PX) * ((g.dh[1] + PY - 1) / PY);
    const int units = tiles * ((n_mtiles + M_CHUNK - 1) / M_CHUNK);
    const int grid = units < nsm ? units : nsm;
    k_corr0_tc<<<grid, THREADS, SMEM, st>>>(g, reinterpret_cast<const __nv_bfloat16*>(a16), d2, lam, pooled0, amax0,
                                           n_mtiles, reinterpret_cast<int*>(status));
    dm_count_launches(2);
    return cudaGetLastError();
}
