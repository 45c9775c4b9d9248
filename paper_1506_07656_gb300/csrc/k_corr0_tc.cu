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
//   B: the implicit im2col of I' for one N-tile of 33 x 7 positions (231 of
//      the 240 rows of the MMA), built in shared memory by all warps in the
//      same layout and kept resident while the CTA sweeps a chunk of M-tiles.
//   D: 128 lanes x 240 FP32 columns of TMEM; two accumulators (columns 0 and
//      256) let the epilogue drain one tile while the next is multiplied.
// Pooling geometry: the N-tile's positions are x = 2 rx0 - 1 + lx (lx < 33),
// y = 2 ry0 - 1 + ly (ly < 7); they cover the 3x3 windows of the 16 x 3
// pooled outputs (rx0 + k, ry0 + j), centre lx = 2k + 1, ly = 2j + 1.
//
// Output path.  P_0 is stored patch-major ([patch][row][pitch]), so the 16
// pooled values of one tile row of one patch are 64 contiguous bytes (16 for
// the argmax codes).  Plain per-thread stores scatter each warp store over 32
// patches (32 sectors per instruction) and saturate L1.  Instead the
// epilogue writes each tile's 128 x 3 x 16 outputs into a shared-memory
// staging buffer (double-buffered) and one thread hands it to the TMA engine
// with two 3-D tensor stores (values, codes); the tensor maps clip rows and
// columns outside the maps and patches past the last one.
//
// Warp roles (576 threads, one CTA per SM, persistent over work units
// (N-tile, M-chunk)): warp 0 issues the bulk copies of A (2-stage ring),
// warp 1 allocates TMEM and one lane issues the MMAs and commits, warps 2-17
// drain the accumulators: four warps per TMEM lane quadrant, each owning four
// of the sixteen pooled columns (C0 columns 8w'..8w'+8) over the three pooled
// rows: 14 tcgen05.ld in three batches of rows (each batch in flight while the
// rows before it are pooled), pool on order-preserving keys that carry the
// position (first maximum in scan order), release the accumulator after the last batch,
// raise to lambda (MUFU-based power), stage, store through TMA.
// FP8 form: the same kernel with E4M3 operands (tcgen05.mma kind::f8f6f4,
// K padded 144 -> 160, five MMAs of K = 32).  Each patch vector is scaled by a
// power of two that brings its largest entry into (224, 448] (E4M3's top
// binade), the image-2 descriptor field by one power of two chosen the same way
// from its largest entry (a grid-wide max reduction first); the epilogue undoes
// both scales per accumulator row before the power.
// Every mbarrier wait is bounded; on timeout the kernel records an error in
// *err, stops issuing work, releases TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "dm_internal.cuh"

#include <memory>

namespace {

constexpr int BM = 128;                       // patches per M-tile (TMEM lanes)
constexpr int KD = 144;                       // 4 x 4 x 9
constexpr int CX = 33, CY = 7;                // C0 positions per N-tile
constexpr int BN = 240;                       // CX * CY = 231, padded to a multiple of 16
constexpr int PX = 16, PY = 3;                // pooled outputs per N-tile
constexpr int EPI_WARPS = 16;
constexpr int EPI_THREADS = 32 * EPI_WARPS;
constexpr int THREADS = 64 + EPI_THREADS;
constexpr int OUT_F = BM * PY * PX * 4;       // 24576: staged values of one tile
constexpr int OUT_C = BM * PY * PX;           // 6144: staged argmax codes of one tile
constexpr long long WAIT_CYCLES = 4000000000LL;     // ~2 s at 2 GHz

enum { FMT_BF16 = 0, FMT_E4M3 = 1 };

// Operand format traits: K padded to the MMA step, bytes per element,
// instruction descriptor (D = F32; A = B = BF16 for kind::f16, E4M3 for kind::f8f6f4),
// and the shared-memory map.
template <int FMT>
struct Fmt {
    static constexpr int KP = FMT == FMT_BF16 ? 144 : 160;
    static constexpr int ESZ = FMT == FMT_BF16 ? 2 : 1;
    static constexpr int KSTEP = FMT == FMT_BF16 ? 16 : 32;
    static constexpr int KSTEPS = KP / KSTEP;
    static constexpr int ROWB = KP * ESZ;              // bytes per operand row
    static constexpr int CHUNKS = ROWB / 16;           // 16-byte core-matrix rows along K
    static constexpr int EPC = 16 / ESZ;               // elements per 16-byte chunk
    static constexpr int GROUP = CHUNKS * 128;         // bytes per 8-row group
    static constexpr int A_TILE = BM * ROWB;
    static constexpr int B_TILE = BN * ROWB;
    static constexpr int STAGES = FMT == FMT_BF16 ? 2 : 3;
    static constexpr int OFF_B = 0;
    static constexpr int OFF_A = ((B_TILE + 1023) / 1024) * 1024;
    static constexpr int OFF_F = ((OFF_A + STAGES * A_TILE + 1023) / 1024) * 1024;
    static constexpr int OFF_C = OFF_F + 2 * OUT_F;
    static constexpr int OFF_BAR = OFF_C + 2 * OUT_C;
    static constexpr size_t SMEM = (size_t)OFF_BAR + 256;
    static constexpr uint32_t IDESC = (1u << 4) | (FMT == FMT_BF16 ? ((1u << 7) | (1u << 10)) : 0u) |
                                      ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
};
static_assert(Fmt<FMT_BF16>::SMEM <= 232448 && Fmt<FMT_E4M3>::SMEM <= 232448, "shared memory");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor, no swizzle: start address,
// leading-dimension byte offset (between core matrices along K), stride byte
// offset (between 8-row groups), fixed field 0b001 at bit 46.
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t group) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((group >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, int* err) {
    long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{.reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p;}"
                     : "=r"(ok) : "r"(bar), "r"(parity), "n"(WAIT_HINT_NS) : "memory");
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

// Three-input maximum (one PTX max with three operands).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ void epi_barrier() { asm volatile("bar.sync 1, %0;" :: "n"(EPI_THREADS) : "memory"); }

// Pack the patch vectors of I into BF16 M-tiles (zero rows past the last patch).
// Rows: image 1's atomic patches (from d1), or the n0 vectors of amat
// (element (dy*4 + dx)*9 + c), zero past the last row.
__global__ void k_pack_a(DmGeom g, const float* __restrict__ d1, __nv_bfloat16* __restrict__ a16, int n_mtiles,
                         const float* __restrict__ amat, int n0) {
    using F = Fmt<FMT_BF16>;
    const long long total = (long long)n_mtiles * BM * F::CHUNKS;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int kc = (int)(idx % F::CHUNKS);
    const int pm = (int)(idx / F::CHUNKS);
    __align__(16) __nv_bfloat16 v[8];
    const int px = 4 * (pm % g.P0x) + 2, py = 4 * (pm / g.P0x) + 2;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        int k = kc * 8 + e;
        int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
        int x = px - 2 + dx, y = py - 2 + dy;
        float f = amat ? (pm < n0 ? __ldg(amat + (long long)pm * KD + k) : 0.0f)
                       : ((pm < n0 && x < g.W1 && y < g.H1) ? __ldg(d1 + ((long long)y * g.W1 + x) * 9 + c) : 0.0f);
        v[e] = __float2bfloat16_rn(f);
    }
    const int t = pm / BM, r = pm % BM;
    char* dst = reinterpret_cast<char*>(a16) + (long long)t * F::A_TILE + (r >> 3) * F::GROUP + kc * 128 + (r & 7) * 16;
    *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
}

// Power of two s with m * s in (224, 448] (E4M3's top binade; 448 = its largest
// finite value), 1 for m = 0.
__device__ __forceinline__ float e4m3_scale(float m) {
    if (!(m > 0.0f)) return 1.0f;
    int e;
    frexpf(448.0f / fmaxf(m, 1e-30f), &e);   // 448/m = f * 2^e, f in [0.5, 1): 2^(e-1) <= 448/m
    return ldexpf(1.0f, e - 1);
}

// Largest |entry| of the image-2 descriptor field, as the bits of a
// non-negative float (monotone as an unsigned integer), into *bmax (zeroed first).
__global__ void k_absmax(const float* __restrict__ d, long long n, unsigned int* __restrict__ bmax) {
    float m = 0.0f;
    const long long n4 = (reinterpret_cast<uintptr_t>(d) & 15) == 0 ? n >> 2 : 0;   // float4 loads only when aligned
    const float4* d4 = reinterpret_cast<const float4*>(d);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = __ldg(d4 + i);
        m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    for (long long i = 4 * n4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(d[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(bmax, __float_as_uint(m));
}

// Pack the patch vectors into E4M3 M-tiles with a per-patch power-of-two scale
// s_p bringing the largest entry into [224, 448]; inv_scale[p] = 1 / s_p.
__global__ void k_pack_a8(DmGeom g, const float* __restrict__ d1, unsigned char* __restrict__ a8,
                          float* __restrict__ inv_scale, int n_mtiles, const float* __restrict__ amat, int n0) {
    using F = Fmt<FMT_E4M3>;
    const int pm = blockIdx.x * blockDim.x + threadIdx.x;
    if (pm >= n_mtiles * BM) return;
    const int px = 4 * (pm % g.P0x) + 2, py = 4 * (pm / g.P0x) + 2;
    float vals[KD];
    float m = 0.0f;
#pragma unroll 4
    for (int k = 0; k < KD; k++) {
        int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
        int x = px - 2 + dx, y = py - 2 + dy;
        float f = amat ? (pm < n0 ? __ldg(amat + (long long)pm * KD + k) : 0.0f)
                       : ((pm < n0 && x < g.W1 && y < g.H1) ? __ldg(d1 + ((long long)y * g.W1 + x) * 9 + c) : 0.0f);
        vals[k] = f;
        m = fmaxf(m, fabsf(f));
    }
    const float s = e4m3_scale(m);
    inv_scale[pm] = 1.0f / s;
    const int t = pm / BM, r = pm % BM;
    char* base = reinterpret_cast<char*>(a8) + (long long)t * F::A_TILE + (r >> 3) * F::GROUP + (r & 7) * 16;
#pragma unroll
    for (int kc = 0; kc < F::CHUNKS; kc++) {
        __align__(16) unsigned char q[16];
#pragma unroll
        for (int e = 0; e < 16; e++) {
            const int k = kc * 16 + e;
            q[e] = k < KD ? (unsigned char)__nv_cvt_float_to_fp8(vals[k] * s, __NV_SATFINITE, __NV_E4M3) : 0;
        }
        *reinterpret_cast<uint4*>(base + kc * 128) = *reinterpret_cast<const uint4*>(q);
    }
}

struct EpiArgs {
    uint32_t taddr;     // TMEM address of this warp's lane quadrant, column 0
    int row;            // accumulator row (patch within the M-tile)
    int part;           // pooled columns 4*part .. 4*part+3
    int cx0, cy0, W2, H2;
    float lam;
    bool interior;      // every C0 position of the N-tile lies inside I'
};

// Accumulator row ly of this thread's part (C0 columns 8 part .. 8 part + 8):
// one 8-column and one 1-column tensor-memory load, completed by the next
// tcgen05.wait::ld.
__device__ __forceinline__ void tmem_row(uint32_t taddr, int ly, uint32_t (&r)[9]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr + ly * CX));
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[8]) : "r"(taddr + ly * CX + 8));
}

// After tcgen05.wait::ld: an empty volatile statement that "rewrites" the row,
// so no use of the loaded registers can be scheduled before the wait.
__device__ __forceinline__ void tmem_row_ready(uint32_t (&r)[9]) {
    asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                      "+r"(r[8]));
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Pooling on order-preserving keys.  An accumulator value is non-negative, so
// its bits order like the value; its 5 low mantissa bits are replaced by 31 -
// (3 ly + c), ly the C0 row (0..6) and c the column (0..8) of this thread's
// block.  Within any 3x3 window (rows 2y..2y+2, columns 2k..2k+2) 3 ly + c is
// the scan-order rank plus the constant 6y + 2k (a column step of at most 2 never
// reaches a row step of 3), so among values equal above those bits the key of
// the position first in scan order is the largest, and the winner's rank is
// (31 - low bits) - (6y + 2k).  The 3x3 maximum of the keys thus gives the
// pooled value (within 31 units of its last place: 2^-18 relative, far below
// the BF16 / E4M3 operand rounding) and its argmax code, with no comparisons.
//
// Horizontal step for C0 row ly: the key maxima of the column triples (2k,
// 2k+1, 2k+2); positions outside I' are -inf.
template <int POS>
__device__ __forceinline__ float pool_key(uint32_t r, uint32_t keep) {
    uint32_t k;
    asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(k) : "r"(r), "r"(keep), "n"(POS));
    return __uint_as_float(k);
}

template <int LY>
__device__ __forceinline__ void pool_row(const EpiArgs& e, int tx0, const uint32_t (&r)[9], float (&h)[4]) {
    // the mask lives in a register, so each key is one three-input logic
    // operation ((r & mask) | position, LUT 0xEA) with the position 31 - (3 ly + c)
    // as its immediate
    uint32_t keep;
    asm("mov.b32 %0, %1;" : "=r"(keep) : "n"(0xFFFFFFE0u));
    float v[9] = {pool_key<31 - 3 * LY>(r[0], keep),     pool_key<31 - 3 * LY - 1>(r[1], keep),
                  pool_key<31 - 3 * LY - 2>(r[2], keep), pool_key<31 - 3 * LY - 3>(r[3], keep),
                  pool_key<31 - 3 * LY - 4>(r[4], keep), pool_key<31 - 3 * LY - 5>(r[5], keep),
                  pool_key<31 - 3 * LY - 6>(r[6], keep), pool_key<31 - 3 * LY - 7>(r[7], keep),
                  pool_key<31 - 3 * LY - 8>(r[8], keep)};
    const int ly = LY;
    if (!e.interior) {
        const int ty = e.cy0 + ly;
        const bool rin = ty >= 0 && ty < e.H2;
#pragma unroll
        for (int c = 0; c < 9; c++) {
            const int tx = tx0 + c;
            if (!(rin && tx >= 0 && tx < e.W2)) v[c] = -INFINITY;
        }
    }
#pragma unroll
    for (int k = 0; k < 4; k++) h[k] = fmax3(v[2 * k], v[2 * k + 1], v[2 * k + 2]);
}

// (a x)^lam = 2^(lam log2 a + lam log2 x) with the hardware's approximate
// base-2 logarithm and exponential, for an accumulator a (never subnormal; 0
// gives 0) and a power-of-two scale x, lc = lam log2 x: one fused multiply-add
// between the two approximations.
__device__ __forceinline__ float pow_hw(float a, float lam, float lc) {
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(a));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(__fmaf_rn(l, lam, lc)));
    return r;
}

// lam log2 x for a power of two x (its exponent field, exactly)
__device__ __forceinline__ float lam_log2_pow2(float x, float lam) {
    return __fmul_rn(lam, (float)((int)((__float_as_uint(x) >> 23) & 0xffu) - 127));
}

// Vertical step for pooled row y (C0 rows 2y, 2y+1, 2y+2 = m_y -1, 0, +1): the
// key maximum, its code 3 (row - 2y) + (c - 2k) from the low bits, the power,
// and the staging of the 4 values and codes.
__device__ __forceinline__ void pool_out(const EpiArgs& e, int y, float lc, const float (&h)[CY][4],
                                         float* stage_f, unsigned char* stage_c) {
    float f[4];
    uint32_t mb[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float m = fmax3(h[2 * y][k], h[2 * y + 1][k], h[2 * y + 2][k]);
        mb[k] = __float_as_uint(m);
        f[k] = pow_hw(m, e.lam, lc);
    }
    // codes 3 row + c - (6 y + 2 k) = (31 - 6 y - 2 k) - (low 5 bits), all four at
    // once: the maxima's low bytes gathered into one word (byte permutes), masked,
    // and subtracted bytewise from the packed constants (no byte borrows: every
    // code is 0..8)
    uint32_t lo01, lo23, lo;
    asm("prmt.b32 %0, %1, %2, 0x0040;" : "=r"(lo01) : "r"(mb[0]), "r"(mb[1]));
    asm("prmt.b32 %0, %1, %2, 0x0040;" : "=r"(lo23) : "r"(mb[2]), "r"(mb[3]));
    asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(lo) : "r"(lo01), "r"(lo23));
    const uint32_t cst = (uint32_t)(31 - 6 * y) * 0x01010101u - 0x06040200u;   // bytes 31 - 6y - 2k
    const uint32_t codes = cst - (lo & 0x1F1F1F1Fu);
    // staging layout = the TMA box [patch][row][16 columns].  The values' box
    // rows (64 bytes, four 16-byte chunks) are staged with the tensor map's
    // 64-byte swizzle: the 16-byte chunk index (shared address bits 4-5) is
    // XORed with address bits 7-8 of the row.  Lanes hold consecutive patches,
    // box rows 3 apart, so without it the 16-byte stores of a quarter warp
    // would hit the same four banks four times.
    const int R = e.row * PY + y;
    const uint32_t row_addr = smem_u32(stage_f) + (uint32_t)R * (PX * 4);
    const int chunk = e.part ^ (int)((row_addr >> 7) & 3u);
    *reinterpret_cast<float4*>(stage_f + R * PX + 4 * chunk) = make_float4(f[0], f[1], f[2], f[3]);
    *reinterpret_cast<uint32_t*>(stage_c + R * PX + 4 * e.part) = codes;
}

// Pool this thread's 4 x 3 outputs of one accumulator, release the
// accumulator, and write the powered values and codes to the staging buffer.
// `mult` turns an accumulator value into C0 (1/16, times the inverse operand
// scales of the FP8 form; positive, so pooling on raw accumulators is exact).
// The seven accumulator rows are read in three batches (rows 0-2, 3-4, 5-6):
// each batch's loads are in flight while the rows before it are pooled, and
// pooled row y is finished as soon as its C0 rows 2y .. 2y+2 are in.
__device__ __forceinline__ void epilogue_tile(const EpiArgs& e, uint32_t b, uint32_t bar_empty, float mult,
                                              float* stage_f, unsigned char* stage_c) {
    const float lc = lam_log2_pow2(mult, e.lam);
    uint32_t r[CY][9];
    float h[CY][4];
    const uint32_t taddr = e.taddr + b * 256 + 8 * e.part;
    const int tx0 = e.cx0 + 8 * e.part;
#pragma unroll
    for (int ly = 0; ly < 3; ly++) tmem_row(taddr, ly, r[ly]);
    tmem_wait();
#pragma unroll
    for (int ly = 0; ly < 3; ly++) tmem_row_ready(r[ly]);
#pragma unroll
    for (int ly = 3; ly < 5; ly++) tmem_row(taddr, ly, r[ly]);
    pool_row<0>(e, tx0, r[0], h[0]);
    pool_row<1>(e, tx0, r[1], h[1]);
    pool_row<2>(e, tx0, r[2], h[2]);
    pool_out(e, 0, lc, h, stage_f, stage_c);
    tmem_wait();
#pragma unroll
    for (int ly = 3; ly < 5; ly++) tmem_row_ready(r[ly]);
#pragma unroll
    for (int ly = 5; ly < 7; ly++) tmem_row(taddr, ly, r[ly]);
    pool_row<3>(e, tx0, r[3], h[3]);
    pool_row<4>(e, tx0, r[4], h[4]);
    pool_out(e, 1, lc, h, stage_f, stage_c);
    tmem_wait();
#pragma unroll
    for (int ly = 5; ly < 7; ly++) tmem_row_ready(r[ly]);
    // every load of this accumulator is complete: hand it back to the MMA warp
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    mbar_arrive(bar_empty);
    pool_row<5>(e, tx0, r[5], h[5]);
    pool_row<6>(e, tx0, r[6], h[6]);
    pool_out(e, 2, lc, h, stage_f, stage_c);
}

// Per-pair arguments of the level-0 kernel.  One launch serves one pair, or
// every pair of a wave of the batched form: the persistent CTAs then drain the
// pairs' work units one after another (pair j owns units first .. first +
// units - 1), keeping the A-tile and accumulator pipelines running across
// pairs; the arguments travel in the kernel parameters, so a captured graph
// replays them as they were.
struct L0Pair {
    CUtensorMap tf, tc;          // pooled values and argmax codes of level 0 (TMA stores)
    DmGeom g;
    const unsigned char* apack;  // packed patch operand (M-tiles)
    const float* inv_sa;         // FP8: inverse per-patch scales
    const unsigned int* bmax;    // FP8: maximum of the image-2 field (float bits)
    const float* d2;             // image-2 descriptors [H2][W2][9]
    int* err;                    // the pair's status word
    int n_mtiles, m_chunk;
    int first, units;
};
struct L0Batch {
    L0Pair p[DM_BATCH_MAX];
    int n, total;
};

template <int FMT>
__global__ void __launch_bounds__(THREADS, 1)
k_corr0_tc(const __grid_constant__ L0Batch B, float lam) {
    using F = Fmt<FMT>;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem + F::OFF_B;
    unsigned char* sA = smem + F::OFF_A;
    float* sF = reinterpret_cast<float*>(smem + F::OFF_F);
    unsigned char* sC = smem + F::OFF_C;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + F::OFF_BAR);
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bars + 2 * F::STAGES + 4);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    const uint32_t bar_full = smem_u32(bars), bar_empty = smem_u32(bars + F::STAGES);
    const uint32_t bar_acc_full = smem_u32(bars + 2 * F::STAGES), bar_acc_empty = smem_u32(bars + 2 * F::STAGES + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < F::STAGES; s++) {
            mbar_init(bar_full + 8 * s, 1);
            mbar_init(bar_empty + 8 * s, 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(bar_acc_full + 8 * b, 1);
            mbar_init(bar_acc_empty + 8 * b, EPI_THREADS);
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

    uint32_t a_it = 0, acc_it = 0;
    const bool store_leader = (warp == 2 && lane == 0);

    for (int gu = blockIdx.x; gu < B.total; gu += gridDim.x) {
        int pj = 0;
        while (pj + 1 < B.n && gu >= B.p[pj + 1].first) pj++;
        const L0Pair& P = B.p[pj];
        const unsigned char* __restrict__ apack = P.apack;
        const float* __restrict__ inv_sa = P.inv_sa;
        const float* __restrict__ d2 = P.d2;
        int* __restrict__ err = P.err;
        const int W2 = P.g.W2, H2 = P.g.H2, mw = P.g.dw[1];
        const int tiles_x = (mw + PX - 1) / PX;
        const int mchunks = (P.n_mtiles + P.m_chunk - 1) / P.m_chunk;
        // image-2 operand scale of the FP8 form (power of two from the field's maximum)
        const float s_b = FMT == FMT_E4M3 ? e4m3_scale(__uint_as_float(*P.bmax)) : 1.0f;
        const int unit = gu - P.first;
        const int m_chunk = P.m_chunk, n_mtiles = P.n_mtiles;
        const int ntile = unit / mchunks, mc = unit % mchunks;
        const int m0 = mc * m_chunk, m1 = min(n_mtiles, m0 + m_chunk), nt = m1 - m0;
        const int rx0 = (ntile % tiles_x) * PX, ry0 = (ntile / tiles_x) * PY;
        const int cx0 = 2 * rx0 - 1, cy0 = 2 * ry0 - 1;

        // B: implicit im2col of I' for this N-tile (zero outside I', past K = 144
        // and in rows 231..239), one 16-byte core-matrix row per item
        for (int ch = tid; ch < BN * F::CHUNKS; ch += THREADS) {
            const int n = ch / F::CHUNKS, kc = ch % F::CHUNKS;
            const int lx = n % CX, ly = n / CX;
            const int tx = cx0 + lx, ty = cy0 + ly;
            uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int e = 0; e < F::EPC; e++) {
                const int k = kc * F::EPC + e;
                const int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
                const int x = tx - 2 + dx, y = ty - 2 + dy;
                const float f = (k < KD && n < CX * CY && x >= 0 && y >= 0 && x < W2 && y < H2)
                                    ? __ldg(d2 + ((long long)y * W2 + x) * 9 + c) : 0.0f;
                if (FMT == FMT_BF16) {
                    w[e >> 1] |= (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f)) << (16 * (e & 1));
                } else {
                    w[e >> 2] |= (uint32_t)__nv_cvt_float_to_fp8(f * s_b, __NV_SATFINITE, __NV_E4M3) << (8 * (e & 3));
                }
            }
            *reinterpret_cast<uint4*>(sB + (n >> 3) * F::GROUP + kc * 128 + (n & 7) * 16) = make_uint4(w[0], w[1], w[2], w[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();

        if (warp == 0) {
            if (lane == 0) {
                for (int j = 0; j < nt; j++) {
                    const uint32_t it = a_it + j, s = it % F::STAGES, ph = (it / F::STAGES) & 1;
                    if (!mbar_wait(bar_empty + 8 * s, ph ^ 1, abort_flag, err)) break;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar_full + 8 * s), "r"(F::A_TILE) : "memory");
                    const unsigned char* src = apack + (long long)(m0 + j) * F::A_TILE;
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(smem_u32(sA + s * F::A_TILE)), "l"(src), "r"(F::A_TILE), "r"(bar_full + 8 * s) : "memory");
                }
            }
        } else if (warp == 1) {
            if (lane == 0) {
                for (int j = 0; j < nt; j++) {
                    const uint32_t it = a_it + j, s = it % F::STAGES, ph = (it / F::STAGES) & 1;
                    const uint32_t ai = acc_it + j, b = ai & 1, aph = (ai >> 1) & 1;
                    if (!mbar_wait(bar_full + 8 * s, ph, abort_flag, err)) break;
                    if (!mbar_wait(bar_acc_empty + 8 * b, aph ^ 1, abort_flag, err)) break;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t d_tmem = tmem + b * 256;
                    const uint32_t a_base = smem_u32(sA + s * F::A_TILE), b_base = smem_u32(sB);
#pragma unroll
                    for (int k = 0; k < F::KSTEPS; k++) {
                        const uint64_t ad = make_desc(a_base + k * 256, F::GROUP), bd = make_desc(b_base + k * 256, F::GROUP);
                        const uint32_t acc = k > 0;
                        if (FMT == FMT_BF16)
                            asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;}"
                                         :: "r"(d_tmem), "l"(ad), "l"(bd), "r"(F::IDESC), "r"(acc) : "memory");
                        else
                            asm volatile("{.reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;}"
                                         :: "r"(d_tmem), "l"(ad), "l"(bd), "r"(F::IDESC), "r"(acc) : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar_empty + 8 * s) : "memory");
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar_acc_full + 8 * b) : "memory");
                }
            }
        } else {
            // epilogue: warp w drains TMEM lane quadrant w % 4, pooled columns of part (w - 2) / 4
            const int quad = warp & 3;
            const EpiArgs ea{tmem + ((uint32_t)(quad * 32) << 16), quad * 32 + lane, (warp - 2) >> 2, cx0, cy0, W2, H2,
                             lam, cx0 >= 0 && cy0 >= 0 && cx0 + CX <= W2 && cy0 + CY <= H2};
            // FP8: 1/16 times the inverse operand scales (powers of two, exact), the
            // patch's scale loaded before the accumulator wait so its latency hides there
            const float mult_b = FMT == FMT_E4M3 ? 0.0625f * (1.0f / s_b) : 0.0625f;
            for (int j = 0; j < nt; j++) {
                const uint32_t ai = acc_it + j, b = ai & 1, aph = (ai >> 1) & 1;
                float mult = mult_b;
                if (FMT == FMT_E4M3) {
                    const int p = (m0 + j) * BM + ea.row;
                    mult = mult_b * __ldg(inv_sa + p);       // inv_sa covers every row of every M-tile
                }
                // a failed (bounded) wait has set the abort flag: this thread skips the
                // tile but still meets the barrier, after which every thread sees the flag
                if (mbar_wait(bar_acc_full + 8 * b, aph, abort_flag, err)) {
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    epilogue_tile(ea, b, bar_acc_empty + 8 * b, mult, sF + b * (OUT_F / 4), sC + b * OUT_C);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                }
                // one barrier per tile: before it the leader also waits until the store
                // of the previous tile has read its staging buffer, which the next tile
                // fills (the staging is double-buffered)
                if (store_leader) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                epi_barrier();
                if (*abort_flag) break;
                float* stf = sF + b * (OUT_F / 4);
                unsigned char* stc = sC + b * OUT_C;
                if (store_leader) {
                    const int z = (m0 + j) * BM;
                    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                                 :: "l"(reinterpret_cast<uint64_t>(&P.tf)), "r"(rx0), "r"(ry0), "r"(z), "r"(smem_u32(stf))
                                 : "memory");
                    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                                 :: "l"(reinterpret_cast<uint64_t>(&P.tc)), "r"(rx0), "r"(ry0), "r"(z), "r"(smem_u32(stc))
                                 : "memory");
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                }
            }
        }
        a_it += nt;
        acc_it += nt;
        __syncthreads();   // the epilogue has consumed every accumulator: the tensor core is done with sB
        if (*abort_flag) break;
    }
    if (store_leader) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(512));
}

// 3-D map of a pooled level-0 array [n0][mh][pitch] (elements of `esize` bytes),
// logical extent mw x mh x n0, box 16 x 3 x 128, staged with the given swizzle.
bool make_map(CUtensorMap* m, void* base, CUtensorMapDataType dt, int esize, const DmGeom& g, int n0, CUtensorMapSwizzle sw) {
    const cuuint64_t dims[3] = {(cuuint64_t)g.dw[1], (cuuint64_t)g.dh[1], (cuuint64_t)n0};
    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch(1) * esize, (cuuint64_t)g.pitch(1) * g.dh[1] * esize};
    const cuuint32_t box[3] = {PX, PY, BM};
    return dm_encode_tiled(m, dt, 3, base, dims, strides, box, sw);
}

template <int FMT>
cudaError_t launch_tc(const L0Batch& B, float lam, cudaStream_t st) {
    using F = Fmt<FMT>;
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    static std::atomic<unsigned long long> smem_done{0};
    cudaError_t ea = dm_smem_opt_in(reinterpret_cast<const void*>(k_corr0_tc<FMT>), (int)F::SMEM, smem_done);
    if (ea != cudaSuccess) return ea;
    if (B.total <= 0) return cudaSuccess;
    const int grid = B.total < nsm ? B.total : nsm;
    k_corr0_tc<FMT><<<grid, THREADS, F::SMEM, st>>>(B, lam);
    return cudaGetLastError();
}

// One pair's entry of a level-0 launch, after its operand packing (launched
// here on st): tensor maps of its outputs, pointers, work units.
cudaError_t prepare_pair(const DmGeom& g, int precision, const float* d1, const float* d2, void* abuf, void* status,
                         float* pooled0, unsigned char* amax0, int m_chunk, cudaStream_t st, const float* amat, int n_rows,
                         L0Pair* q) {
    memset(q, 0, sizeof(*q));
    const int n0 = n_rows < 0 ? g.npatch(0) : n_rows;
    const int n_mtiles = (n0 + BM - 1) / BM;
    if (m_chunk < 1) m_chunk = 1;
    // values: 64-byte box rows staged with the 64-byte swizzle (see pool_out)
    if (!make_map(&q->tf, pooled0, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g, n0, CU_TENSOR_MAP_SWIZZLE_64B) ||
        !make_map(&q->tc, amax0, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, g, n0, CU_TENSOR_MAP_SWIZZLE_NONE))
        return cudaErrorNotSupported;
    unsigned char* apack = reinterpret_cast<unsigned char*>(abuf);
    q->g = g;
    q->apack = apack;
    q->d2 = d2;
    q->err = reinterpret_cast<int*>(status);
    q->n_mtiles = n_mtiles;
    q->m_chunk = m_chunk;
    q->units = ((g.dw[1] + PX - 1) / PX) * ((g.dh[1] + PY - 1) / PY) * ((n_mtiles + m_chunk - 1) / m_chunk);
    cudaError_t e;
    if (precision == DM_FP8_E4M3) {
        const size_t a_bytes = dm_align((size_t)n_mtiles * Fmt<FMT_E4M3>::A_TILE);
        float* inv_sa = reinterpret_cast<float*>(apack + a_bytes);
        unsigned int* bmax = reinterpret_cast<unsigned int*>(apack + a_bytes + dm_align((size_t)n_mtiles * BM * sizeof(float)));
        if ((e = cudaMemsetAsync(bmax, 0, sizeof(unsigned int), st)) != cudaSuccess) return e;
        const long long n2 = (long long)g.W2 * g.H2 * 9;
        const long long blocks = (n2 / 4 + 255) / 256;
        k_absmax<<<(unsigned)(blocks < 1216 ? (blocks > 0 ? blocks : 1) : 1216), 256, 0, st>>>(d2, n2, bmax);
        k_pack_a8<<<(unsigned)((n_mtiles * BM + 127) / 128), 128, 0, st>>>(g, d1, apack, inv_sa, n_mtiles, amat, n0);
        q->inv_sa = inv_sa;
        q->bmax = bmax;
        dm_count_launches(2);
    } else {
        long long total = (long long)n_mtiles * BM * Fmt<FMT_BF16>::CHUNKS;
        k_pack_a<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(g, d1, reinterpret_cast<__nv_bfloat16*>(apack), n_mtiles,
                                                                   amat, n0);
        dm_count_launches(1);
    }
    return cudaGetLastError();
}

}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool dm_encode_tiled(CUtensorMap* m, CUtensorMapDataType dt, int rank, void* base, const cuuint64_t* dims,
                     const cuuint64_t* strides_bytes, const cuuint32_t* box, CUtensorMapSwizzle swizzle) {
    // looked up once (thread-safe initialisation of a function-local static)
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<EncodeTiledFn>(p);
        return nullptr;
    }();
    if (!fn) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(m, dt, (cuuint32_t)rank, base, dims, strides_bytes, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              swizzle, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Packed-operand buffer: A tiles; FP8 form also the per-patch inverse scales
// (f32 [n_mtiles * 128]) and the image-2 maximum (one u32).
size_t dm_corr0_tc_a_bytes(const DmGeom& g, int precision) {
    const size_t n_mtiles = ((size_t)g.npatch(0) + BM - 1) / BM;
    if (precision == DM_FP8_E4M3)
        return dm_align(n_mtiles * Fmt<FMT_E4M3>::A_TILE) + dm_align(n_mtiles * BM * sizeof(float)) + sizeof(unsigned int);
    return n_mtiles * Fmt<FMT_BF16>::A_TILE;
}

cudaError_t dm_launch_corr0_tc(const DmGeom& g, int precision, const float* d1, const float* d2, float lam, void* abuf,
                               void* status, float* pooled0, unsigned char* amax0, int m_chunk, cudaStream_t st,
                               const float* amat, int n_rows) {
    std::unique_ptr<L0Batch> B(new L0Batch);
    memset(B.get(), 0, sizeof(L0Batch));
    cudaError_t e = prepare_pair(g, precision, d1, d2, abuf, status, pooled0, amax0, m_chunk, st, amat, n_rows, &B->p[0]);
    if (e != cudaSuccess) return e;
    B->n = 1;
    B->total = B->p[0].units;
    e = precision == DM_FP8_E4M3 ? launch_tc<FMT_E4M3>(*B, lam, st) : launch_tc<FMT_BF16>(*B, lam, st);
    dm_count_launches(1);
    return e;
}

cudaError_t dm_launch_corr0_tc_batch(int n, const DmGeom* gs, int precision, const float* const* d1s,
                                     const float* const* d2s, float lam, void* const* abufs, void* const* statuses,
                                     float* const* pooled0s, unsigned char* const* amax0s, const int* m_chunks,
                                     cudaStream_t st) {
    if (n < 1 || n > DM_BATCH_MAX) return cudaErrorInvalidValue;
    std::unique_ptr<L0Batch> B(new L0Batch);
    memset(B.get(), 0, sizeof(L0Batch));
    for (int j = 0; j < n; j++) {
        cudaError_t e = prepare_pair(gs[j], precision, d1s[j], d2s[j], abufs[j], statuses[j], pooled0s[j], amax0s[j],
                                     m_chunks[j], st, nullptr, -1, &B->p[j]);
        if (e != cudaSuccess) return e;
        B->p[j].first = B->total;
        B->total += B->p[j].units;
    }
    B->n = n;
    cudaError_t e = precision == DM_FP8_E4M3 ? launch_tc<FMT_E4M3>(*B, lam, st) : launch_tc<FMT_BF16>(*B, lam, st);
    dm_count_launches(1);
    return e;
}
