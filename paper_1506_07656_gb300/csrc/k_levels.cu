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
// This pass streams the pooled maps of the level below and does a fixed
// amount of arithmetic per stored output (~4 averages of 4 values, a 9-way
// max with argmax, one power).  A CTA owns a tile of 32 x TH pooled outputs
// (TH = 8 by default on 4 warps; 16 on 8 or 4 on 2, autotuned) of a run of up
// to 32 lattice patches on one row,
// spaced so that the right child column of one patch is the left child column
// of the next: the child windows (72 x (2 TH + 1) floats, which cover both
// shifts +-1 of a shared column) are staged in shared memory by 3-D TMA tensor
// loads into a ring of NR = 2 (or 3, autotuned) columns; as soon as a patch's
// averages are formed its left column is released and one thread starts the
// loads of the column NR ahead, which overlap the pooling and rectification.
// Each child window reaches shared memory about twice per (up to) four parents
// instead of four times; the CTAs of one tile row and one row of patches run
// together, so the second staging (by the next row of patches) and the window
// edges shared by neighbouring tiles come from L2, and the maps are read from
// DRAM about 1.1 times.
// Every thread forms the same number of averages and of pooled outputs per
// patch (the CTA meets a barrier after each phase).
// (Rows of the pooled maps are padded to 16 floats and the window's first
// column is a multiple of 4, so every load starts 16-byte aligned; the tensor
// map zero-fills whatever lies outside the domain.)  Algorithmic bytes per
// stored output: 16 B of child values read (each child value is shared by 4
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

// Three-input maximum (one PTX max with three operands).
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

constexpr int TW = 32;                           // pooled columns per CTA tile (one per lane)
constexpr int AW = 2 * TW + 1;                   // average columns per CTA (65)
constexpr int KW = 72;                           // staged child columns (TMA box width)
constexpr int AWP = 68;                          // padded row of the averages (16-byte aligned rows)
constexpr int LEVEL_THREADS = 256;
// threads of a tiled level CTA for TH pooled rows: 8 warps for 16 rows, 4 for 8,
// 2 for 4 -- every thread forms two 4-column average groups and two pooled
// outputs per patch, and smaller CTAs wait less at their per-patch barriers
// (1024x436 levels: 8 rows on 4 warps 7.79 ms, 16 rows on 8 warps 8.30, 8 rows
// on 8 warps 10.31)
template <int TH>
__host__ __device__ constexpr int level_threads() { return TH == 16 ? 256 : (TH == 8 ? 128 : 64); }

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

// Averages at staged row ay, columns ax .. ax+3 of child 0's frame, from the
// four child windows (a missing child's window holds zeros, which leave both
// the plain and the compensated sum of the others unchanged: s + 0 = s exactly,
// with a zero TwoSum error): child i contributes its column ax + o_x,i + 3.
// Children with o_x = -1 (left, windows lt / lb) read columns ax+2 .. ax+5 (two
// aligned float4 loads, which unlike 8-byte loads at a 16-byte stride are free
// of bank conflicts), children with o_x = +1 (right, rt / rb) columns
// ax+4 .. ax+7.  Then times w (1/n for n = 1, 2, 4, exact) or, for n = 3,
// divided by 3.  Two columns per packed FP32x2 operation: Knuth's TwoSum (6
// additions, every step correctly rounded per lane) costs 3 instructions per
// column and step.
template <bool COMP, bool DIV3>
__device__ __forceinline__ float2 avg_pair4(float2 x0, float2 x1, float2 x2, float2 x3, float w) {
    float2 sv = x0;
    if constexpr (COMP) {
        float2 cp, err;
        // first step: the compensation starts as its error term (0 + err = err;
        // a -0 there would only meet s + (+-0) = s at the end)
        dm_two_sum2(sv, x1, cp);
        dm_two_sum2(sv, x2, err);
        cp = __fadd2_rn(cp, err);
        dm_two_sum2(sv, x3, err);
        cp = __fadd2_rn(cp, err);
        sv = __fadd2_rn(sv, cp);
    } else {
        sv = __fadd2_rn(__fadd2_rn(__fadd2_rn(sv, x1), x2), x3);
    }
    return DIV3 ? make_float2(__fdiv_rn(sv.x, 3.0f), __fdiv_rn(sv.y, 3.0f)) : __fmul2_rn(sv, make_float2(w, w));
}

template <bool COMP, bool DIV3>
__device__ __forceinline__ float4 avg_group(const float* lt, const float* lb, const float* rt, const float* rb, float w) {
    const float4 a0 = *reinterpret_cast<const float4*>(lt), b0 = *reinterpret_cast<const float4*>(lt + 4);
    const float4 a1 = *reinterpret_cast<const float4*>(lb), b1 = *reinterpret_cast<const float4*>(lb + 4);
    const float4 v2 = *reinterpret_cast<const float4*>(rt + 4);
    const float4 v3 = *reinterpret_cast<const float4*>(rb + 4);
    const float2 r0 = avg_pair4<COMP, DIV3>(make_float2(a0.z, a0.w), make_float2(a1.z, a1.w), make_float2(v2.x, v2.y),
                                            make_float2(v3.x, v3.y), w);
    const float2 r1 = avg_pair4<COMP, DIV3>(make_float2(b0.x, b0.y), make_float2(b1.x, b1.y), make_float2(v2.z, v2.w),
                                            make_float2(v3.z, v3.w), w);
    return make_float4(r0.x, r0.y, r1.x, r1.y);
}

// The same for two columns c, c+1 (c even: 8-byte loads at columns c+2 and
// c+4), or -- ONE -- for column c alone (the second lane's result unused).
template <bool COMP, bool DIV3, bool ONE>
__device__ __forceinline__ float2 avg_two(const float* lt, const float* lb, const float* rt, const float* rb, float w) {
    float2 x[4];
    if constexpr (ONE) {
        x[0] = make_float2(lt[2], 0.0f);
        x[1] = make_float2(lb[2], 0.0f);
        x[2] = make_float2(rt[4], 0.0f);
        x[3] = make_float2(rb[4], 0.0f);
    } else {
        x[0] = *reinterpret_cast<const float2*>(lt + 2);
        x[1] = *reinterpret_cast<const float2*>(lb + 2);
        x[2] = *reinterpret_cast<const float2*>(rt + 4);
        x[3] = *reinterpret_cast<const float2*>(rb + 4);
    }
    return avg_pair4<COMP, DIV3>(x[0], x[1], x[2], x[3], w);
}

// Sweep geometry of level l: a CTA owns one tile of TW x TH pooled outputs of a
// run of `run` lattice patches on one row iy, ix = r + (k0 + k) * S.  Patch ix
// has its children in the lattice (or atomic-grid) columns ix - d and ix + d'
// of level l-1 (level 1: ix - 1 and ix; level l >= 2: ix -+ 2^(l-2)), rows
// iy - e, iy + e' likewise; the stride S = 2^(l-1) (1 at level 1) makes the
// right column of one patch the left column of the next, so the run needs
// run + 1 columns of two child windows each instead of 4 windows per patch.
// Runs of 32 (measured at 1024x436 with 8-row tiles, levels stage: 8 8.09 ms,
// 16 7.79, 32 7.66, 48 7.67, 64 7.63; 32 keeps more CTAs for small images;
// shorter runs on the small top levels gained nothing).
__host__ __device__ inline int level_run(int) { return 32; }

__device__ __forceinline__ void child_col_row(const DmGeom& g, int l, int ix, int iy, int* cx_left, int* cy_top, int* step) {
    if (l == 1) { *cx_left = ix - 1; *cy_top = iy - 1; *step = 1; }
    else { const int s = 1 << (l - 2); *cx_left = ix - s; *cy_top = iy - s; *step = 2 * s; }
}

// Index at level l-1 of the child at column cx, row cy, or -1 (outside the
// grid, or not existing).
__device__ __forceinline__ int child_at(const DmGeom& g, int l, int cx, int cy, const unsigned char* __restrict__ vprev) {
    const int gx = l == 1 ? g.P0x : g.Lx, gy = l == 1 ? g.P0y : g.Ly;
    if (cx < 0 || cy < 0 || cx >= gx || cy >= gy) return -1;
    const int c = cy * gx + cx;
    return vprev[c] ? c : -1;
}

// Level l in [1, L-1].  Work item = (tile row, row iy, tile column, residue r,
// run k0) with the residue and run fastest, so the CTAs whose windows overlap
// (neighbouring runs, neighbouring tiles of a tile row, and -- one row of
// patches later -- the rows that share child windows) run close together in
// time.  `tmap` maps the pooled maps of
// level l-1 as a 3-D array (columns dw[l], rows dh[l], patches) with a
// 72 x (2 TH + 1) x 1 box.  Dynamic shared memory: a ring of NR columns x 2
// child windows, then the averages.  Per patch of the run: form the averages
// from its two columns, release the left column (thread 0 starts the loads of
// the column NR ahead into it), pool, power, store, wait for the next patch's
// columns; two barriers per patch.
template <bool COMP, int TH, int NR, bool APPROX, int NT = LEVEL_THREADS>
__device__ __forceinline__ void level_sweep_body(const DmGeom& g, int l, const CUtensorMap* tmap_p,
                                                 const unsigned char* __restrict__ vprev, int runs_per_res, int run,
                                                 float* __restrict__ out, unsigned char* __restrict__ amax, float lam,
                                                 int* __restrict__ err, const int* __restrict__ proto_of, int n_maps,
                                                 long long inject_wait, int item) {
    using T = LevelTile<TH>;
    constexpr int AH = T::AH, KIDF = T::KIDF;
    extern __shared__ __align__(128) unsigned char lsm_raw[];
    // TMA destinations must be 128-byte aligned: round the dynamic base up (128 bytes are reserved for this)
    float* lsm = reinterpret_cast<float*>(lsm_raw + ((128u - ((uint32_t)__cvta_generic_to_shared(lsm_raw) & 127u)) & 127u));
    float* ring = lsm;                                       // [NR][2][KIDF]
    float (*avg)[AWP] = reinterpret_cast<float (*)[AWP]>(lsm + NR * 2 * KIDF);
    __shared__ __align__(8) uint64_t bars[NR + 1];          // ring slots, then one barrier nothing completes
    __shared__ int colc[NR][2];                              // child index per ring slot (top, bottom), -1 absent
    __shared__ int abort_s;

    const int ow = g.dw[l + 1], oh = g.dh[l + 1], opitch = g.pitch(l + 1);
    const int mw = g.dw[l], mh = g.dh[l];
    const int tiles_x = (ow + TW - 1) / TW;
    int cx0, cy0, S;
    child_col_row(g, l, 0, 0, &cx0, &cy0, &S);
    const int per_row = S * runs_per_res;
    // work item = (tile row, lattice row iy, tile column, run): the CTAs of one
    // tile row and one row of patches run together, so the window edges that
    // neighbouring tiles of the row share (64-byte memory granules at their x
    // edges) come from DRAM once, and the next row of patches, which stages the
    // same child rows again, follows within a few hundred CTAs, while they are
    // still in L2 (1024x436, level 1: DRAM reads 1.14x the maps; all tiles of a
    // row of patches together instead: 2.1x, their child rows exceed the L2
    // before the next row of patches reads them again; the tile as the slowest
    // index: 1.83x at 512x224)
    const int rr = item % per_row;
    int t = item / per_row;
    const int tx = t % tiles_x;
    t /= tiles_x;
    const int iy = t % g.Ly;
    const int tile = (t / g.Ly) * tiles_x + tx;
    const int r = rr / runs_per_res, k0 = (rr - r * runs_per_res) * run;
    const int ix0 = r + k0 * S;                              // first patch of the run
    if (ix0 >= g.Lx) return;
    const int nrun = min(run, (g.Lx - 1 - ix0) / S + 1);    // patches in this run
    const int rx0 = (tile % tiles_x) * TW, ry0 = (tile / tiles_x) * TH;
    const int qx0 = 2 * rx0 - 1, qy0 = 2 * ry0 - 1;
    const int xa = 2 * rx0 - 4;                              // first staged child column (multiple of 4 floats)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int cxl, cyt, st;
    child_col_row(g, l, ix0, iy, &cxl, &cyt, &st);
    const int cyb = cyt + (l == 1 ? 1 : S);                  // bottom child row

    // start the loads of column j (child column cxl + j*S) into slot j % NR (one thread);
    // a missing child's window is loaded from map index -1, outside the tensor,
    // which the TMA unit fills with zeros without reading memory
    auto stage = [&](int j) {
        const int slot = j % NR;
        const int cx = cxl + j * S;
        const int ct = child_at(g, l, cx, cyt, vprev), cb = child_at(g, l, cx, cyb, vprev);
        colc[slot][0] = ct;
        colc[slot][1] = cb;
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[slot]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(2u * T::KID_BYTES) : "memory");
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(ring + slot * 2 * KIDF);
        // the map of an atomic child is its prototype's in the approximate form
        int zt = ct, zb = cb;
        if constexpr (APPROX) {
            // (an entry outside [0, maps) would only read the zero fill; it is
            // clamped like everywhere else)
            if (ct >= 0) zt = min(max(__ldg(proto_of + ct), 0), n_maps - 1);
            if (cb >= 0) zb = min(max(__ldg(proto_of + cb), 0), n_maps - 1);
        }
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                     :: "r"(dst), "l"(reinterpret_cast<uint64_t>(tmap_p)), "r"(xa), "r"(qy0 - 1), "r"(zt), "r"(bar)
                     : "memory");
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                     :: "r"(dst + KIDF * 4), "l"(reinterpret_cast<uint64_t>(tmap_p)), "r"(xa), "r"(qy0 + 1), "r"(zb), "r"(bar)
                     : "memory");
    };
    // wait for column j (the (j / NR)-th use of its slot); false on timeout
    auto wait_col = [&](int j) -> bool {
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[j % NR]);
        const uint32_t parity = (uint32_t)((j / NR) & 1);
        const long long t0 = clock64();
        while (true) {
            uint32_t done;
            asm volatile("{.reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3; selp.u32 %0, 1, 0, q;}"
                         : "=r"(done) : "r"(bar), "r"(parity), "n"(WAIT_HINT_NS) : "memory");
            if (done) return true;
            if (clock64() - t0 > LEVEL_WAIT_CYCLES) return false;
        }
    };

    if (tid == 0) {
        abort_s = 0;
        for (int b = 0; b <= NR; b++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"((uint32_t)__cvta_generic_to_shared(&bars[b])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int j = 0; j < NR && j <= nrun; j++) stage(j);
        if (inject_wait > 0) {
            // fault injection: a bounded wait on a barrier nothing completes runs
            // out after inject_wait cycles, exactly like a wait for a load that
            // never lands; the CTA then takes its abort path below (which still
            // waits, with the normal limit, for the loads it has started)
            const uint32_t never = (uint32_t)__cvta_generic_to_shared(&bars[NR]);
            const long long t0 = clock64();
            uint32_t done = 0;
            while (!done && clock64() - t0 <= inject_wait)
                asm volatile("{.reg .pred q; mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3; selp.u32 %0, 1, 0, q;}"
                             : "=r"(done) : "r"(never), "r"(0u), "n"(WAIT_HINT_NS) : "memory");
            if (!done) { atomicOr(err, 1); abort_s = 1; }
        }
    }
    __syncthreads();
    const bool interior = qx0 >= 0 && qy0 >= 0 && qx0 + AW <= mw && qy0 + AH <= mh;
    // thread 0 waits for the loads; the barrier after its wait passes their
    // data on to every thread of the CTA
    if (tid == 0 && (!wait_col(0) || !wait_col(1))) { atomicOr(err, 1); abort_s = 1; }
    __syncthreads();                                         // columns 0, 1 and their colc visible; abort agreed
    for (int k = 0; k < nrun; k++) {
        if (abort_s) {
            // let the loads already started finish (each wait bounded) before the CTA exits
            if (tid == 0)
                for (int j = k; j <= min(k + NR - 1, nrun); j++) wait_col(j);
            return;
        }
        const int sl = k % NR, sr = (k + 1) % NR;
        const int ci[4] = {colc[sl][0], colc[sl][1], colc[sr][0], colc[sr][1]};
        const int n = (ci[0] >= 0) + (ci[1] >= 0) + (ci[2] >= 0) + (ci[3] >= 0);
        const int ix = ix0 + k * S;
        const int p = iy * g.Lx + ix;
        if (n > 0) {
            // averages of the tile: rows 0 .. 2 TH - 1 in 16 groups of 4 columns
            // (columns 0 .. 63), 32 TH / NT groups per thread; then the last row's 32
            // column pairs and column 64 of every row, one item each for threads
            // from 64 on.  (A tile that reaches past the map holds -inf at the
            // positions outside the domain, which the pooling then never selects.)
            const float* lt = ring + (sl * 2) * KIDF;
            const float* rt = ring + (sr * 2) * KIDF;
            const float w = n == 4 ? 0.25f : (n == 2 ? 0.5f : 1.0f);
            auto mask = [&](float& v, int ay, int ax) {
                const int qy = qy0 + ay, qx = qx0 + ax;
                if (qy < 0 || qy >= mh || qx < 0 || qx >= mw) v = -INFINITY;
            };
#pragma unroll
            for (int u = 0; u < 32 * TH / NT; u++) {
                const int e = tid + u * NT;
                const int ay = e >> 4, ax = 4 * (e & 15);
                const int o = ay * KW + ax;
                float4 a = n == 3 ? avg_group<COMP, true>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w)
                                  : avg_group<COMP, false>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w);
                if (!interior) {
                    mask(a.x, ay, ax);
                    mask(a.y, ay, ax + 1);
                    mask(a.z, ay, ax + 2);
                    mask(a.w, ay, ax + 3);
                }
                *reinterpret_cast<float4*>(&avg[ay][ax]) = a;
            }
            constexpr int XB = NT >= 64 + 32 + AH ? 64 : NT - (32 + AH);   // first thread of the extra items
            const int x = tid - XB;
            if (x >= 0 && x < 32 + AH) {
                if (x < 32) {
                    // last row, columns 2x, 2x + 1
                    const int ay = AH - 1, ax = 2 * x, o = ay * KW + ax;
                    float2 a = n == 3 ? avg_two<COMP, true, false>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w)
                                      : avg_two<COMP, false, false>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w);
                    if (!interior) {
                        mask(a.x, ay, ax);
                        mask(a.y, ay, ax + 1);
                    }
                    *reinterpret_cast<float2*>(&avg[ay][ax]) = a;
                } else {
                    // column 64 of row x - 32
                    const int ay = x - 32, ax = AW - 1, o = ay * KW + ax;
                    float2 a = n == 3 ? avg_two<COMP, true, true>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w)
                                      : avg_two<COMP, false, true>(lt + o, lt + KIDF + o, rt + o, rt + KIDF + o, w);
                    if (!interior) mask(a.x, ay, ax);
                    avg[ay][ax] = a.x;
                }
            }
        }
        __syncthreads();                                     // averages ready; column k no longer needed
        // into the slot column k just released; issued from the last warp, so that
        // warp 0, whose thread 0 waits for the loads, does not carry both
        if (tid == NT - 32 && k + NR <= nrun) stage(k + NR);
        if (n > 0) {
            // 3x3 / 2 max-pool over in-domain averages, first strict maximum, power.
            // A thread owns R = 32 TH / NT vertically adjacent outputs (rows R*warp ..), so
            // the horizontal 3-maxima of the 2R+1 average rows it reads are formed
            // once (a row shared by two outputs serves both); rows are then merged in
            // scan order m_y = -1, 0, 1, which keeps the first strict maximum.
            constexpr int R = 32 * TH / NT;
            static_assert(R >= 1 && 32 + AH <= NT && 32 * TH % NT == 0, "tile rows and threads");
            const int rx = rx0 + lane;
            const int ty0 = R * warp;
            if (rx < ow) {
                float hv[2 * R + 1], h0[2 * R + 1], h1[2 * R + 1];
#pragma unroll
                for (int kk = 0; kk < 2 * R + 1; kk++) {
                    const int ay = 2 * ty0 + kk;             // average row; map row qy0 + ay
                    const float a0 = avg[ay][2 * lane], a1 = avg[ay][2 * lane + 1], a2 = avg[ay][2 * lane + 2];
                    hv[kk] = fmax3(a0, a1, a2);
                    h0[kk] = a0;
                    h1[kk] = a1;
                }
                float best[R], pw[R];
                int code[R];
#pragma unroll
                for (int j = 0; j < R; j++) {
                    // first row holding the maximum (m_y = -1, 0, 1), then the first column of
                    // that row holding it (m_x = -1, 0, 1): the first maximum in scan order
                    best[j] = fmax3(hv[2 * j], hv[2 * j + 1], hv[2 * j + 2]);
                    const bool r0 = hv[2 * j] == best[j], r1 = hv[2 * j + 1] == best[j];
                    const float x0 = r0 ? h0[2 * j] : (r1 ? h0[2 * j + 1] : h0[2 * j + 2]);
                    const float x1 = r0 ? h1[2 * j] : (r1 ? h1[2 * j + 1] : h1[2 * j + 2]);
                    code[j] = (r0 ? 0 : (r1 ? 3 : 6)) + (x0 == best[j] ? 0 : (x1 == best[j] ? 1 : 2));
                }
                // the power of two outputs per packed evaluation (rows past the map
                // are evaluated on whatever the tile holds there and not stored)
#pragma unroll
                for (int j = 0; j + 1 < R; j += 2) {
                    const float2 v = dm_powf2(make_float2(best[j], best[j + 1]), lam);
                    pw[j] = v.x;
                    pw[j + 1] = v.y;
                }
                if constexpr (R % 2 == 1) pw[R - 1] = dm_powf(best[R - 1], lam);
#pragma unroll
                for (int j = 0; j < R; j++) {
                    const int ry = ry0 + ty0 + j;
                    if (ry >= oh) break;
                    const long long o = ((long long)p * oh + ry) * opitch + rx;
                    out[o] = pw[j];
                    amax[o] = (unsigned char)code[j];
                }
            }
        }
        // the next patch's columns k+1, k+2 (waited for by thread 0), then one
        // barrier: averages consumed, those columns and their colc visible, abort agreed
        if (tid == 0 && k + 1 < nrun && (!wait_col(k + 1) || !wait_col(k + 2))) { atomicOr(err, 1); abort_s = 1; }
        __syncthreads();
    }
}

template <bool COMP, int TH, int NR, bool APPROX = false, int NT = level_threads<TH>()>
__global__ void __launch_bounds__(NT) k_level_sweep(DmGeom g, int l, const __grid_constant__ CUtensorMap tmap,
                                                               const unsigned char* __restrict__ vprev,
                                                               int runs_per_res, int run, float* __restrict__ out,
                                                               unsigned char* __restrict__ amax, float lam,
                                                               int* __restrict__ err, const int* __restrict__ proto_of,
                                                               int n_maps, long long inject_wait) {
    level_sweep_body<COMP, TH, NR, APPROX, NT>(g, l, &tmap, vprev, runs_per_res, run, out, amax, lam, err, proto_of, n_maps,
                                               inject_wait, (int)blockIdx.x);
}

// ---------------------------------------------------------------------------
// Row-streaming form of the same pass (level_th = 0 in the tuned shapes).
//
// One warp owns one lattice patch p and a strip of STREAM_W = 31 pooled columns
// [r0, r0 + 31) of its stored map, and walks down every row of it: no shared
// memory, no barrier.  For a row y of averages, lane t forms A(2(r0+t) - 1, y)
// and A(2(r0+t), y), two columns at once with the packed child sum: the
// children with o_x = -1 contribute their columns 2(r0+t) - 2 and - 1, those
// with o_x = +1 their columns 2(r0+t) and + 1 -- one aligned 8-byte load per
// child, from row y - 1 (o_y = -1) or y + 1 (o_y = +1).  A(2(r0+t) + 1, y) is
// lane t+1's first average (one shuffle); lane 31 only supplies it.  The
// horizontal 3-maxima of the rows stay in registers and merge over three rows
// into the pooled output, two output rows per step (one packed power).
// Missing children and samples outside the domain read as 0, which leaves both
// child sums unchanged (s + 0 = s exactly, with a zero TwoSum error), so every
// patch runs the four-child arithmetic and divides by its number of children;
// warps whose strip and children lie wholly inside take loads without any
// masks, and only the first and last steps check rows.  The 8 warps of a CTA
// take a 4 x 2 block of patches spaced S apart, which share child maps: each
// child row a CTA needs comes from L2 once and is reused from L1.
// ---------------------------------------------------------------------------
constexpr int STREAM_W = 31;        // pooled columns per warp strip
constexpr int STREAM_BX = 4, STREAM_BY = 2;   // patches per CTA along x and y
constexpr int STREAM_WARPS = STREAM_BX * STREAM_BY;

// Average of the four children (child order i = 0..3, zeros for missing ones)
// for two columns at once, then times 1/n (n = 3 divides).
template <bool COMP>
__device__ __forceinline__ float2 avg_pair(const float2* v, int n) {
    float2 sv = v[0];
    if constexpr (COMP) {
        float2 cp = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int i = 1; i < 4; i++) {
            float2 err;
            dm_two_sum2(sv, v[i], err);
            cp = i == 1 ? err : __fadd2_rn(cp, err);
        }
        sv = __fadd2_rn(sv, cp);
    } else {
#pragma unroll
        for (int i = 1; i < 4; i++) sv = __fadd2_rn(sv, v[i]);
    }
    if (n == 4) return __fmul2_rn(sv, make_float2(0.25f, 0.25f));
    if (n == 3) return make_float2(__fdiv_rn(sv.x, 3.0f), __fdiv_rn(sv.y, 3.0f));
    const float w = n == 2 ? 0.5f : 1.0f;
    return __fmul2_rn(sv, make_float2(w, w));
}

// Per-warp state of the row-streaming kernel.
struct StreamWarp {
    const float* kid[4];   // child maps (nullptr: missing)
    int n;                 // existing children
    int mw, mh, pitch;     // child map domain and row pitch (level l)
    int xl, xr;            // first column of this lane's left / right child pairs
    int ml, mr;            // their load modes: 3 both columns in the domain, 1 only the first, 0 none
    bool has_a0, has_a2;   // A(2rx - 1) and A(2rx + 1) in the domain
};

// The four children's pairs of A row y.  CHECK: rows outside the domain, missing
// children and columns outside the domain read as zeros; otherwise every load is
// known to be inside.
template <bool CHECK>
__device__ __forceinline__ void stream_load_row(const StreamWarp& w, float2* v, int y) {
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int cy = y + ((i & 1) ? 1 : -1);
        const int x = i < 2 ? w.xl : w.xr;
        if constexpr (!CHECK) {
            v[i] = __ldg(reinterpret_cast<const float2*>(w.kid[i] + (cy * w.pitch + x)));
        } else {
            const int mode = i < 2 ? w.ml : w.mr;
            const bool ok = w.kid[i] != nullptr && cy >= 0 && cy < w.mh;
            float2 t = make_float2(0.0f, 0.0f);
            if (ok && mode == 3) t = __ldg(reinterpret_cast<const float2*>(w.kid[i] + (cy * w.pitch + x)));
            else if (ok && mode == 1) t.x = __ldg(w.kid[i] + (cy * w.pitch + x));
            v[i] = t;
        }
    }
}

// Horizontal 3-max (first column equal to the maximum) of A row y; -inf outside the domain.
template <bool COMP>
__device__ __forceinline__ void stream_hrow(const StreamWarp& w, const float2* v, int y, float& h, int& hc) {
    const float2 a = avg_pair<COMP>(v, w.n);
    const float a2s = __shfl_down_sync(0xffffffffu, a.x, 1);
    const float a0 = w.has_a0 ? a.x : -INFINITY, a1 = a.y, a2 = w.has_a2 ? a2s : -INFINITY;
    const float m = fmax3(a0, a1, a2);
    h = y < w.mh ? m : -INFINITY;
    hc = a0 == m ? 0 : (a1 == m ? 1 : 2);
}

// One step: output rows ry and ry + 1 from A rows 2ry - 1 (carried in hp, cp)
// to 2ry + 3.
template <bool COMP, bool CHECK>
__device__ __forceinline__ void stream_step(const StreamWarp& w, int ry, int oh, float& hp, int& cp, float lam,
                                            bool store, float* __restrict__ orow, unsigned char* __restrict__ arow,
                                            int opitch) {
    float2 v[4][4];
#pragma unroll
    for (int k = 0; k < 4; k++) stream_load_row<CHECK>(w, v[k], 2 * ry + k);
    float h[4];
    int hc[4];
#pragma unroll
    for (int k = 0; k < 4; k++) stream_hrow<COMP>(w, v[k], 2 * ry + k, h[k], hc[k]);
    const float b0 = fmax3(hp, h[0], h[1]);
    const int c0 = hp == b0 ? cp : (h[0] == b0 ? 3 + hc[0] : 6 + hc[1]);
    const float b1 = fmax3(h[1], h[2], h[3]);
    const int c1 = h[1] == b1 ? hc[1] : (h[2] == b1 ? 3 + hc[2] : 6 + hc[3]);
    hp = h[3];
    cp = hc[3];
    const bool two = ry + 1 < oh;
    // (with one output row left, the second lane of the pair repeats the first and is not stored)
    const float2 pw = dm_powf2(make_float2(b0, two ? b1 : b0), lam);
    if (store) {
        orow[(long long)ry * opitch] = pw.x;
        arow[(long long)ry * opitch] = (unsigned char)c0;
        if (two) {
            orow[(long long)(ry + 1) * opitch] = pw.y;
            arow[(long long)(ry + 1) * opitch] = (unsigned char)c1;
        }
    }
}

template <bool COMP, bool APPROX>
__device__ __forceinline__ void level_stream_body(const DmGeom& g, int l, const float* __restrict__ prev,
                                                  const unsigned char* __restrict__ vprev,
                                                  const unsigned char* __restrict__ vcur, int bx_per_res, int by_per_res,
                                                  float* __restrict__ out, unsigned char* __restrict__ amax, float lam,
                                                  const int* __restrict__ proto_of, int n_maps, long long item) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cx0, cy0, S;
    child_col_row(g, l, 0, 0, &cx0, &cy0, &S);
    // block = (((strip * S + res_y) * by_per_res + by) * S + res_x) * bx_per_res + bx: a block holds
    // patches (res_x + (bx * 4 + wx) S, res_y + (by * 2 + wy) S), wx < 4, wy < 2
    const int bx = (int)(item % bx_per_res);
    item /= bx_per_res;
    const int res_x = (int)(item % S);
    item /= S;
    const int by = (int)(item % by_per_res);
    item /= by_per_res;
    const int res_y = (int)(item % S);
    const int strip = (int)(item / S);
    const int ix = res_x + (bx * STREAM_BX + (warp % STREAM_BX)) * S;
    const int iy = res_y + (by * STREAM_BY + (warp / STREAM_BX)) * S;
    if (ix >= g.Lx || iy >= g.Ly) return;
    const int p = iy * g.Lx + ix;
    if (!vcur[p]) return;

    StreamWarp w;
    w.mw = g.dw[l];
    w.mh = g.dh[l];
    w.pitch = g.pitch(l);
    const int ow = g.dw[l + 1], oh = g.dh[l + 1], opitch = g.pitch(l + 1);
    const long long csize = g.psize(l);
    w.n = 0;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int c = dm_child(g, l, ix, iy, i);
        w.kid[i] = nullptr;
        if (c >= 0 && vprev[c]) {
            const int cm = APPROX ? min(max(__ldg(proto_of + c), 0), n_maps - 1) : c;
            w.kid[i] = prev + (long long)cm * csize;
            w.n++;
        }
    }
    const int r0 = strip * STREAM_W, rx = r0 + lane;
    w.xl = 2 * rx - 2;
    w.xr = 2 * rx;
    auto mode_of = [&](int x) { return (x >= 0 && x < w.mw) ? ((x + 1 < w.mw) ? 3 : 1) : 0; };
    w.ml = mode_of(w.xl);
    w.mr = mode_of(w.xr);
    w.has_a0 = rx >= 1;
    w.has_a2 = 2 * rx + 1 < w.mw;
    const bool store = lane < STREAM_W && rx < ow;
    // every lane's pairs inside the domain and all four children present
    const bool inside = w.n == 4 && 2 * r0 - 2 >= 0 && 2 * (r0 + 31) + 1 < w.mw;

    float* orow = out + (long long)p * oh * opitch + rx;
    unsigned char* arow = amax + (long long)p * oh * opitch + rx;
    float hp = -INFINITY;                                   // A row 2ry - 1 (none for ry = 0)
    int cp = 0;
    int ry = 0;
    if (inside) {
        // step ry reads child rows 2ry - 1 .. 2ry + 4: unchecked while they lie in the domain
        stream_step<COMP, true>(w, 0, oh, hp, cp, lam, store, orow, arow, opitch);
        for (ry = 2; 2 * ry + 4 < w.mh; ry += 2) stream_step<COMP, false>(w, ry, oh, hp, cp, lam, store, orow, arow, opitch);
    }
    for (; ry < oh; ry += 2) stream_step<COMP, true>(w, ry, oh, hp, cp, lam, store, orow, arow, opitch);
}

template <bool COMP, bool APPROX = false>
__global__ void __launch_bounds__(STREAM_WARPS * 32, 4) k_level_stream(DmGeom g, int l, const float* __restrict__ prev,
                                                                   const unsigned char* __restrict__ vprev,
                                                                   const unsigned char* __restrict__ vcur,
                                                                   int bx_per_res, int by_per_res, float* __restrict__ out,
                                                                   unsigned char* __restrict__ amax, float lam,
                                                                   const int* __restrict__ proto_of, int n_maps) {
    level_stream_body<COMP, APPROX>(g, l, prev, vprev, vcur, bx_per_res, by_per_res, out, amax, lam, proto_of, n_maps,
                                    (long long)blockIdx.x);
}

// Top level L: C_L = (mean of children)^lambda over the domain of level L.
template <bool COMP>
__global__ void k_level_top(DmGeom g, int l, const unsigned char* __restrict__ vprev,
                            const unsigned char* __restrict__ vcur, const float* __restrict__ prev,
                            float* __restrict__ top, float lam, const int* __restrict__ proto_of, int n_maps) {
    const int p = blockIdx.y;
    if (!vcur[p]) return;
    const int mw = g.dw[l], mh = g.dh[l];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= mw * mh) return;
    Kids k;
    load_kids(g, l, p, vprev, prev, k, proto_of, n_maps);
    float a = child_mean<COMP>(k, q % mw, q / mw, mw, mh, g.pitch(l));
    top[(long long)p * mw * mh + q] = dm_powf(a, lam);
}

template <bool COMP, int TH, int NR, bool APPROX = false, int NT = level_threads<TH>()>
cudaError_t launch_sweep(const DmGeom& g, int l, const CUtensorMap& tm, const dm_pyramid& py, int per_res, long long items,
                         float lam, int* status, cudaStream_t st) {
    const size_t smem = (size_t)(NR * 2 * LevelTile<TH>::KIDF + LevelTile<TH>::AH * AWP) * sizeof(float) + 128;
    static std::atomic<unsigned long long> smem_done{0};
    cudaError_t ea = dm_smem_opt_in(reinterpret_cast<const void*>(k_level_sweep<COMP, TH, NR, APPROX, NT>), (int)smem, smem_done);
    if (ea != cudaSuccess) return ea;
    if (items <= 0) return cudaSuccess;
    if (items > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_level_sweep<COMP, TH, NR, APPROX, NT><<<(unsigned)items, NT, smem, st>>>(g, l, tm, py.valid[l - 1], per_res, level_run(l),
                                                                          const_cast<float*>(py.pooled[l]),
                                                                          const_cast<unsigned char*>(py.amax[l]), lam, status,
                                                                          APPROX ? py.proto_of : nullptr, py.n0_maps,
                                                                          py.inject_wait);
    return cudaGetLastError();
}

template <bool COMP, bool APPROX = false>
cudaError_t launch_stream(const DmGeom& g, int l, const dm_pyramid& py, float lam, cudaStream_t st) {
    const int S = l == 1 ? 1 : 1 << (l - 1);
    const int bx_per_res = ((g.Lx + S - 1) / S + STREAM_BX - 1) / STREAM_BX;
    const int by_per_res = ((g.Ly + S - 1) / S + STREAM_BY - 1) / STREAM_BY;
    const int strips = (g.dw[l + 1] + STREAM_W - 1) / STREAM_W;
    const long long blocks = (long long)strips * S * by_per_res * S * bx_per_res;
    if (blocks <= 0) return cudaSuccess;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_level_stream<COMP, APPROX><<<(unsigned)blocks, STREAM_WARPS * 32, 0, st>>>(
        g, l, py.pooled[l - 1], py.valid[l - 1], py.valid[l], bx_per_res, by_per_res, const_cast<float*>(py.pooled[l]),
        const_cast<unsigned char*>(py.amax[l]), lam, APPROX ? py.proto_of : nullptr, py.n0_maps);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cross-pair form: one launch per step of the pass for every pair of a wave
// of the batched form (dm_launch_levels_batch).  The per-pair arguments travel
// in the kernel parameters (a captured graph replays them as they were), and
// block b of a launch belongs to the pair j with first[j] <= b < first[j+1]
// (tiled and row-streaming kernels) or to pair blockIdx.y / blockIdx.z.
// ---------------------------------------------------------------------------
struct LvPair {
    CUtensorMap tmap;          // tiled kernel: the pooled maps of level l-1
    DmGeom g;
    const unsigned char* vprev;
    unsigned char* vcur;
    const float* prev;         // pooled maps of level l-1
    float* out;                // pooled maps of level l (or the top)
    unsigned char* amax;
    int* err;
    int a, b;                  // tiled: runs per residue; row-streaming: blocks per residue in x, y
    long long first;           // first block of this pair in the launch
};
struct LvBatch {
    LvPair p[DM_BATCH_MAX];
    int n;
};

__device__ __forceinline__ int lv_pair_of(const LvBatch& B, long long blk) {
    int j = 0;
    while (j + 1 < B.n && blk >= B.p[j + 1].first) j++;
    return j;
}

template <bool COMP, int TH, int NR>
__global__ void __launch_bounds__(level_threads<TH>()) k_level_sweep_b(const __grid_constant__ LvBatch B, int l, float lam) {
    const int j = lv_pair_of(B, blockIdx.x);
    const LvPair& P = B.p[j];
    level_sweep_body<COMP, TH, NR, false, level_threads<TH>()>(P.g, l, &P.tmap, P.vprev, P.a, level_run(l), P.out, P.amax,
                                                               lam, P.err, nullptr, 0, 0,
                                                               (int)((long long)blockIdx.x - P.first));
}

template <bool COMP>
__global__ void __launch_bounds__(STREAM_WARPS * 32, 4) k_level_stream_b(const __grid_constant__ LvBatch B, int l, float lam) {
    const int j = lv_pair_of(B, blockIdx.x);
    const LvPair& P = B.p[j];
    level_stream_body<COMP, false>(P.g, l, P.prev, P.vprev, P.vcur, P.a, P.b, P.out, P.amax, lam, nullptr, 0,
                                   (long long)blockIdx.x - P.first);
}

__global__ void k_valid_b(const __grid_constant__ LvBatch B, int l) {
    const LvPair& P = B.p[blockIdx.y];
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (l == 0) {
        if (p < P.g.npatch(0)) P.vcur[p] = 1;
        return;
    }
    if (p >= P.g.Lx * P.g.Ly) return;
    const int ix = p % P.g.Lx, iy = p / P.g.Lx;
    unsigned char any = 0;
    for (int i = 0; i < 4; i++) {
        const int c = dm_child(P.g, l, ix, iy, i);
        if (c >= 0 && P.vprev[c]) any = 1;
    }
    P.vcur[p] = any;
}

template <bool COMP>
__global__ void k_level_top_b(const __grid_constant__ LvBatch B, int l, float lam) {
    const LvPair& P = B.p[blockIdx.z];
    const DmGeom& g = P.g;
    const int p = blockIdx.y;
    if (p >= g.npatch(l) || !P.vcur[p]) return;
    const int mw = g.dw[l], mh = g.dh[l];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= mw * mh) return;
    Kids k;
    load_kids(g, l, p, P.vprev, P.prev, k, nullptr, g.npatch(0));
    const float a = child_mean<COMP>(k, q % mw, q / mw, mw, mh, g.pitch(l));
    P.out[(long long)p * mw * mh + q] = dm_powf(a, lam);
}

}  // namespace

cudaError_t dm_launch_levels(const DmGeom& g, const dm_pyramid& py, float lam, int* status, cudaStream_t st) {
    const int B = 128;
    int n0 = g.npatch(0), np = g.npatch(1);
    k_fill_u8<<<(n0 + 255) / 256, 256, 0, st>>>(const_cast<unsigned char*>(py.valid[0]), n0, 1);
    for (int l = 1; l <= g.L; l++) {
        k_valid<<<(np + 255) / 256, 256, 0, st>>>(g, l, py.valid[l - 1], const_cast<unsigned char*>(py.valid[l]));
        // the row-streaming kernel: as the tuned shape, and always for the levels
        // whose stored maps are at most 16 columns wide, where the tiled kernel's
        // per-patch pipeline is latency-bound (1024x436: levels 5-7 take 0.18
        // instead of 0.38 ms); a fault-injection run takes the tiled kernel,
        // which holds the bounded waits
        const bool stream = py.tune.level_th == 0 || g.dw[l + 1] <= 16;
        if (l < g.L && stream && py.inject_wait == 0) {
            const bool approx = l == 1 && py.proto_of != nullptr;
            cudaError_t e;
            if (approx)
                e = py.compensated ? launch_stream<true, true>(g, l, py, lam, st) : launch_stream<false, true>(g, l, py, lam, st);
            else
                e = py.compensated ? launch_stream<true>(g, l, py, lam, st) : launch_stream<false>(g, l, py, lam, st);
            if (e != cudaSuccess) return e;
        } else if (l < g.L) {
            // pooled maps of level l-1: [npatch(l-1)][dh[l]][pitch(l)] floats
            // level 1 of an approximate pyramid reads the level-0 maps through the
            // prototype index: its own kernel instance, 16-row tiles, ring of 2
            const bool approx = l == 1 && py.proto_of != nullptr;
            const int th = approx ? 16 : (py.tune.level_th == 8 || py.tune.level_th == 4 ? py.tune.level_th : 16);
            CUtensorMap tm;
            // (level 0 holds n0_maps maps: one per atomic patch, or per prototype)
            const cuuint64_t dims[3] = {(cuuint64_t)g.dw[l], (cuuint64_t)g.dh[l],
                                        (cuuint64_t)(l == 1 ? py.n0_maps : g.npatch(l - 1))};
            const cuuint64_t strides[2] = {(cuuint64_t)g.pitch(l) * 4, (cuuint64_t)g.psize(l) * 4};
            const cuuint32_t box[3] = {KW, (cuuint32_t)(2 * th + 1), 1};
            if (!dm_encode_tiled(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(py.pooled[l - 1]), dims,
                                 strides, box))
                return cudaErrorNotSupported;
            const int tiles = ((g.dw[l + 1] + TW - 1) / TW) * ((g.dh[l + 1] + th - 1) / th);
            const int S = l == 1 ? 1 : 1 << (l - 1);
            const int run = level_run(l);
            const int per_res = ((g.Lx + S - 1) / S + run - 1) / run;    // runs per residue class
            const long long items = (long long)tiles * g.Ly * S * per_res;
            cudaError_t e;
            const bool r2 = py.tune.level_ring == 2;
            if (approx)
                e = py.compensated ? launch_sweep<true, 16, 2, true>(g, l, tm, py, per_res, items, lam, status, st)
                                   : launch_sweep<false, 16, 2, true>(g, l, tm, py, per_res, items, lam, status, st);
            else if (th == 8)
                e = py.compensated ? (r2 ? launch_sweep<true, 8, 2> : launch_sweep<true, 8, 3>)(g, l, tm, py, per_res, items, lam, status, st)
                                   : (r2 ? launch_sweep<false, 8, 2> : launch_sweep<false, 8, 3>)(g, l, tm, py, per_res, items, lam, status, st);
            else if (th == 4)
                e = py.compensated ? (r2 ? launch_sweep<true, 4, 2> : launch_sweep<true, 4, 3>)(g, l, tm, py, per_res, items, lam, status, st)
                                   : (r2 ? launch_sweep<false, 4, 2> : launch_sweep<false, 4, 3>)(g, l, tm, py, per_res, items, lam, status, st);
            else
                e = py.compensated ? (r2 ? launch_sweep<true, 16, 2> : launch_sweep<true, 16, 3>)(g, l, tm, py, per_res, items, lam, status, st)
                                   : (r2 ? launch_sweep<false, 16, 2> : launch_sweep<false, 16, 3>)(g, l, tm, py, per_res, items, lam, status, st);
            if (e != cudaSuccess) return e;
        } else {
            int n = g.dw[l] * g.dh[l];
            dim3 grid((n + B - 1) / B, np);
            auto kern = py.compensated ? k_level_top<true> : k_level_top<false>;
            kern<<<grid, B, 0, st>>>(g, l, py.valid[l - 1], py.valid[l], py.pooled[l - 1], const_cast<float*>(py.top), lam,
                                     l == 1 ? py.proto_of : nullptr, py.n0_maps);
        }
    }
    dm_count_launches(1 + 2 * g.L);
    return cudaGetLastError();
}

// Levels >= 1 of the n <= DM_BATCH_MAX pyramids of a wave (level 0 computed):
// per level, one launch of the existence flags and one launch per kernel shape
// in use (tiled with each tuned (rows, ring), row-streaming, top) for all the
// pairs at that level; status[j] receives pair j's bounded-wait flag.
cudaError_t dm_launch_levels_batch(const dm_pyramid* const* pys, int n, float lam, int* const* status, cudaStream_t st) {
    if (n < 1 || n > DM_BATCH_MAX) return cudaErrorInvalidValue;
    const bool comp = pys[0]->compensated != 0;
    int Lmax = 0;
    for (int j = 0; j < n; j++) Lmax = max(Lmax, pys[j]->g.L);
    long long launches = 0;
    auto base_pair = [&](int j, int l) {
        const dm_pyramid& py = *pys[j];
        LvPair q;
        memset(&q, 0, sizeof(q));
        q.g = py.g;
        q.vprev = l >= 1 ? py.valid[l - 1] : nullptr;
        q.vcur = const_cast<unsigned char*>(py.valid[l]);
        q.prev = l >= 1 ? py.pooled[l - 1] : nullptr;
        q.out = l < py.g.L ? const_cast<float*>(py.pooled[l]) : const_cast<float*>(py.top);
        q.amax = l < py.g.L ? const_cast<unsigned char*>(py.amax[l]) : nullptr;
        q.err = status[j];
        return q;
    };
    for (int l = 0; l <= Lmax; l++) {
        // existence flags of level l (level 0: every atomic patch)
        {
            LvBatch B;
            memset(&B, 0, sizeof(B));
            int maxp = 0;
            for (int j = 0; j < n; j++)
                if (l <= pys[j]->g.L) {
                    B.p[B.n++] = base_pair(j, l);
                    maxp = max(maxp, pys[j]->g.npatch(l));
                }
            if (B.n == 0) break;
            k_valid_b<<<dim3((unsigned)((maxp + 255) / 256), (unsigned)B.n), 256, 0, st>>>(B, l);
            launches++;
        }
        if (l == 0) continue;
        // the pairs whose level l is the top
        {
            LvBatch B;
            memset(&B, 0, sizeof(B));
            int maxq = 0, maxp = 0;
            for (int j = 0; j < n; j++)
                if (l == pys[j]->g.L) {
                    B.p[B.n++] = base_pair(j, l);
                    maxq = max(maxq, pys[j]->g.dw[l] * pys[j]->g.dh[l]);
                    maxp = max(maxp, pys[j]->g.npatch(l));
                }
            if (B.n) {
                const dim3 grid((unsigned)((maxq + 127) / 128), (unsigned)maxp, (unsigned)B.n);
                if (comp) k_level_top_b<true><<<grid, 128, 0, st>>>(B, l, lam);
                else k_level_top_b<false><<<grid, 128, 0, st>>>(B, l, lam);
                launches++;
            }
        }
        // the pairs below their top: one launch per kernel shape in use.
        // shape 0: row-streaming; 1 + 2 (rows 16 / 8 / 4 as 0 / 1 / 2) + (ring == 3): tiled
        for (int shape = 0; shape < 7; shape++) {
            LvBatch B;
            memset(&B, 0, sizeof(B));
            long long blocks = 0;
            for (int j = 0; j < n; j++) {
                const dm_pyramid& py = *pys[j];
                const DmGeom& g = py.g;
                if (l >= g.L) continue;
                const bool stream = py.tune.level_th == 0 || g.dw[l + 1] <= 16;
                const int th = py.tune.level_th == 8 || py.tune.level_th == 4 ? py.tune.level_th : 16;
                const int nr = py.tune.level_ring == 3 ? 3 : 2;
                const int my = stream ? 0 : 1 + 2 * (th == 16 ? 0 : (th == 8 ? 1 : 2)) + (nr == 3);
                if (my != shape) continue;
                LvPair q = base_pair(j, l);
                const int S = l == 1 ? 1 : 1 << (l - 1);
                long long items;
                if (stream) {
                    q.a = ((g.Lx + S - 1) / S + STREAM_BX - 1) / STREAM_BX;
                    q.b = ((g.Ly + S - 1) / S + STREAM_BY - 1) / STREAM_BY;
                    const int strips = (g.dw[l + 1] + STREAM_W - 1) / STREAM_W;
                    items = (long long)strips * S * q.b * S * q.a;
                } else {
                    const cuuint64_t dims[3] = {(cuuint64_t)g.dw[l], (cuuint64_t)g.dh[l], (cuuint64_t)g.npatch(l - 1)};
                    const cuuint64_t strides[2] = {(cuuint64_t)g.pitch(l) * 4, (cuuint64_t)g.psize(l) * 4};
                    const cuuint32_t box[3] = {KW, (cuuint32_t)(2 * th + 1), 1};
                    if (!dm_encode_tiled(&q.tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(py.pooled[l - 1]),
                                         dims, strides, box))
                        return cudaErrorNotSupported;
                    const int tiles = ((g.dw[l + 1] + TW - 1) / TW) * ((g.dh[l + 1] + th - 1) / th);
                    const int run = level_run(l);
                    q.a = ((g.Lx + S - 1) / S + run - 1) / run;
                    items = (long long)tiles * g.Ly * S * q.a;
                }
                q.first = blocks;
                blocks += items;
                B.p[B.n++] = q;
            }
            if (B.n == 0 || blocks == 0) continue;
            if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
            cudaError_t e = cudaSuccess;
            if (shape == 0) {
                if (comp) k_level_stream_b<true><<<(unsigned)blocks, STREAM_WARPS * 32, 0, st>>>(B, l, lam);
                else k_level_stream_b<false><<<(unsigned)blocks, STREAM_WARPS * 32, 0, st>>>(B, l, lam);
            } else {
                auto launch = [&](auto kern, int TH, int NR) -> cudaError_t {
                    const int kidf = (((2 * TH + 1) * KW + 31) / 32) * 32;     // LevelTile<TH>::KIDF
                    const size_t smem = (size_t)(NR * 2 * kidf + (2 * TH + 1) * AWP) * sizeof(float) + 128;
                    const int nt = TH == 16 ? level_threads<16>() : (TH == 8 ? level_threads<8>() : level_threads<4>());
                    static std::atomic<unsigned long long> done[6];
                    cudaError_t ea = dm_smem_opt_in(reinterpret_cast<const void*>(kern), (int)smem, done[shape - 1]);
                    if (ea != cudaSuccess) return ea;
                    kern<<<(unsigned)blocks, nt, smem, st>>>(B, l, lam);
                    return cudaSuccess;
                };
                switch (shape) {
                    case 1: e = comp ? launch(k_level_sweep_b<true, 16, 2>, 16, 2) : launch(k_level_sweep_b<false, 16, 2>, 16, 2); break;
                    case 2: e = comp ? launch(k_level_sweep_b<true, 16, 3>, 16, 3) : launch(k_level_sweep_b<false, 16, 3>, 16, 3); break;
                    case 3: e = comp ? launch(k_level_sweep_b<true, 8, 2>, 8, 2) : launch(k_level_sweep_b<false, 8, 2>, 8, 2); break;
                    case 4: e = comp ? launch(k_level_sweep_b<true, 8, 3>, 8, 3) : launch(k_level_sweep_b<false, 8, 3>, 8, 3); break;
                    case 5: e = comp ? launch(k_level_sweep_b<true, 4, 2>, 4, 2) : launch(k_level_sweep_b<false, 4, 2>, 4, 2); break;
                    default: e = comp ? launch(k_level_sweep_b<true, 4, 3>, 4, 3) : launch(k_level_sweep_b<false, 4, 3>, 4, 3); break;
                }
            }
            if (e != cudaSuccess) return e;
            launches++;
        }
    }
    dm_count_launches(launches);
    return cudaGetLastError();
}
