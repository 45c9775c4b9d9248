// Approximate DeepMatching (Sec. 4.1): the prototype dictionary.
//
// The atomic patches of image 1 (144-vectors, the Eq. 3-4 window, zero
// outside the image) are clustered by k-means with every centroid projected
// back on the hypersphere of the patches (norm 4: 16 unit pixel descriptors)
// after each update; each patch is then replaced by its closest prototype, so
// the bottom level needs one correlation map per prototype instead of one per
// patch (dm_correlate_pyramid_approx).
//
// One iteration = assignment, then update:
//   assignment: the closest centroid = the largest dot product (all centroids
//     have the same norm), ties to the lower index.  k_km_assign fuses the
//     P0 x D x 144 product with the running argmax: a CTA stages 128 patch
//     vectors in shared memory once and streams the centroids in tiles of 64;
//     each dot product is one fma chain over k = 0..143 in FP32.
//   update: each centroid = the sum of its members projected to norm 4 (a
//     centroid without members keeps its value).  The member sums are exact
//     and independent of the order of arrival: every entry (in [0, 1]) is
//     rounded to a multiple of 2^-40 and added as a 64-bit integer, so the
//     result does not depend on atomic ordering; the norm and the projection
//     are computed in FP64 and rounded to FP32 once.
// A final assignment pairs the patches with the returned prototypes.
#include "dm_internal.cuh"

namespace {

constexpr int KM_BM = 128;     // patches per CTA of the assignment
constexpr int KM_BN = 64;      // centroids per tile
constexpr int ASTR = KM_BM + 4;   // shared row strides (16-byte multiples, fewer bank conflicts on the transposing stores)
constexpr int CSTR = KM_BN + 4;
constexpr int KD = 144;
constexpr double FIX = 1099511627776.0;   // 2^40

__global__ void k_patch_vectors(DmGeom g, const float* __restrict__ d1, float* __restrict__ A) {
    const long long n = (long long)g.P0x * g.P0y * KD;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int p = (int)(idx / KD), k = (int)(idx % KD);
    const int dy = k / 36, dx = (k / 9) % 4, c = k % 9;
    const int x = 4 * (p % g.P0x) + dx, y = 4 * (p / g.P0x) + dy;    // centre - 2 + offset
    A[idx] = (x < g.W1 && y < g.H1) ? __ldg(d1 + ((long long)y * g.W1 + x) * 9 + c) : 0.0f;
}

// Sum over the threads of a block (blockDim.x a multiple of 32, <= 1024).
__device__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < nw; i++) t += red[i];
    return t;
}

// C[d] = A[init[d]] projected to norm 4 (unchanged if zero).
__global__ void k_km_init(const float* __restrict__ A, const int* __restrict__ init, float* __restrict__ C) {
    __shared__ double red[32];
    const int d = blockIdx.x, k = threadIdx.x;
    const float a = k < KD ? A[(long long)init[d] * KD + k] : 0.0f;
    const double nn = block_sum((double)a * a, red);
    if (k < KD) C[(long long)d * KD + k] = nn > 0.0 ? (float)((double)a * (4.0 / sqrt(nn))) : a;
}

__device__ __forceinline__ bool better(float s, int i, float bs, int bi) { return s > bs || (s == bs && i < bi); }

// The best centroid of chunk blockIdx.y (centroids [y*chunk, (y+1)*chunk))
// for each patch: (score, index) into part_s / part_i [gridDim.y][P0].  A
// CTA holds 128 patch vectors (As[144][132]) and streams its centroids in
// tiles of 64 (Cs[144][68]); a thread owns 8 patches x 4 centroids of each
// tile (vector shared loads, 32 fmas per 3 loads) and keeps its patches'
// running best.
__global__ void __launch_bounds__(256) k_km_assign(const float* __restrict__ A, int P0, const float* __restrict__ C, int D,
                                                   int chunk, float* __restrict__ part_s, int* __restrict__ part_i) {
    extern __shared__ __align__(16) float kms[];
    float* As = kms;                       // [KD][ASTR]
    float* Cs = kms + KD * ASTR;           // [KD][CSTR]
    const int tid = threadIdx.x, p0 = blockIdx.x * KM_BM;
    // staged transposed; the global reads run along k (coalesced)
    for (int e = tid; e < KD * KM_BM; e += 256) {
        const int m = e / KD, k = e - m * KD;
        As[k * ASTR + m] = p0 + m < P0 ? A[(long long)(p0 + m) * KD + k] : 0.0f;
    }
    const int tm = (tid % 16) * 8, tn = (tid / 16) * 4;
    float best[8];
    int bidx[8];
#pragma unroll
    for (int i = 0; i < 8; i++) { best[i] = -INFINITY; bidx[i] = 0x7fffffff; }
    const int nb = blockIdx.y * chunk, ne = min(D, nb + chunk);
    for (int n0 = nb; n0 < ne; n0 += KM_BN) {
        __syncthreads();
        for (int e = tid; e < KD * KM_BN; e += 256) {
            const int n = e / KD, k = e - n * KD;
            Cs[k * CSTR + n] = n0 + n < ne ? C[(long long)(n0 + n) * KD + k] : 0.0f;
        }
        __syncthreads();
        float acc[8][4] = {};
#pragma unroll 2
        for (int k = 0; k < KD; k++) {
            const float4 a0 = *reinterpret_cast<const float4*>(As + k * ASTR + tm);
            const float4 a1 = *reinterpret_cast<const float4*>(As + k * ASTR + tm + 4);
            const float4 b = *reinterpret_cast<const float4*>(Cs + k * CSTR + tn);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = __fmaf_rn(av[i], bv[j], acc[i][j]);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int d = n0 + tn + j;
            if (d >= ne) continue;
#pragma unroll
            for (int i = 0; i < 8; i++)
                if (better(acc[i][j], d, best[i], bidx[i])) { best[i] = acc[i][j]; bidx[i] = d; }
        }
    }
    // the 16 threads holding the same 8 patches (different centroid columns) agree
    __syncthreads();
    float* rs = Cs;                                          // [16][KM_BM]
    int* ri = reinterpret_cast<int*>(Cs + 16 * KM_BM);       // [16][KM_BM]
#pragma unroll
    for (int i = 0; i < 8; i++) {
        rs[(tid / 16) * KM_BM + tm + i] = best[i];
        ri[(tid / 16) * KM_BM + tm + i] = bidx[i];
    }
    __syncthreads();
    if (tid < KM_BM && p0 + tid < P0) {
        float bs = rs[tid];
        int bi = ri[tid];
        for (int j = 1; j < 16; j++)
            if (better(rs[j * KM_BM + tid], ri[j * KM_BM + tid], bs, bi)) { bs = rs[j * KM_BM + tid]; bi = ri[j * KM_BM + tid]; }
        part_s[(long long)blockIdx.y * P0 + p0 + tid] = bs;
        part_i[(long long)blockIdx.y * P0 + p0 + tid] = bi;
    }
}

// assign[p] = the best of the chunks' candidates (same order rule: the larger
// score, then the lower index), so the split does not change the result.
__global__ void k_km_merge(const float* __restrict__ part_s, const int* __restrict__ part_i, int P0, int nchunk, int D,
                           int* __restrict__ assign) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P0) return;
    float bs = part_s[p];
    int bi = part_i[p];
    for (int y = 1; y < nchunk; y++)
        if (better(part_s[(long long)y * P0 + p], part_i[(long long)y * P0 + p], bs, bi)) {
            bs = part_s[(long long)y * P0 + p];
            bi = part_i[(long long)y * P0 + p];
        }
    assign[p] = bi < D ? bi : 0;                             // (no finite score at all: prototype 0)
}

// S[d][k] += A[p][k] in 2^-40 fixed point, cnt[d] += 1, for d = assign[p].
__global__ void k_km_accum(const float* __restrict__ A, long long n, const int* __restrict__ assign,
                           unsigned long long* __restrict__ S, unsigned int* __restrict__ cnt) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const int p = (int)(idx / KD), k = (int)(idx % KD);
    const int d = assign[p];
    const unsigned long long v = __double2ull_rn((double)A[idx] * FIX);
    if (v) atomicAdd(S + (long long)d * KD + k, v);
    if (k == 0) atomicAdd(cnt + d, 1u);
}

// C[d] = S[d] projected to norm 4, if the cluster has members.
__global__ void k_km_finish(const unsigned long long* __restrict__ S, const unsigned int* __restrict__ cnt,
                            float* __restrict__ C) {
    __shared__ double red[32];
    const int d = blockIdx.x, k = threadIdx.x;
    if (cnt[d] == 0) return;                                 // uniform over the block
    const double s = k < KD ? (double)S[(long long)d * KD + k] * (1.0 / FIX) : 0.0;
    const double nn = block_sum(s * s, red);
    if (k < KD && nn > 0.0) C[(long long)d * KD + k] = (float)(s * (4.0 / sqrt(nn)));
}

struct KmLayout {
    size_t A, S, cnt, init, part_s, part_i, bytes;
    int nchunk, chunk;
};

KmLayout km_layout(const DmGeom& g, int D) {
    KmLayout l;
    size_t o = 0;
    l.A = o;    o += dm_align((size_t)g.P0x * g.P0y * KD * sizeof(float));
    l.S = o;    o += dm_align((size_t)D * KD * sizeof(unsigned long long));
    l.cnt = o;  o += dm_align((size_t)D * sizeof(unsigned int));
    l.init = o; o += dm_align((size_t)D * sizeof(int));
    // centroid chunks: enough CTAs for about three waves of two per SM on 152 SMs
    const int P0 = g.P0x * g.P0y;
    const int mblocks = (P0 + KM_BM - 1) / KM_BM;
    const int want = (912 + mblocks - 1) / mblocks;
    const int maxc = (D + KM_BN - 1) / KM_BN;
    const int nsplit = want < 1 ? 1 : (want > maxc ? maxc : want);
    l.chunk = (((D + nsplit - 1) / nsplit) + KM_BN - 1) / KM_BN * KM_BN;
    l.nchunk = (D + l.chunk - 1) / l.chunk;
    l.part_s = o; o += dm_align((size_t)l.nchunk * P0 * sizeof(float));
    l.part_i = o; o += dm_align((size_t)l.nchunk * P0 * sizeof(int));
    l.bytes = o;
    return l;
}

}  // namespace

size_t dm_kmeans_ws_bytes(const DmGeom& g, int D) { return km_layout(g, D).bytes; }

// `init` is a device array of D patch indices (already validated) inside ws.
cudaError_t dm_launch_kmeans(const DmGeom& g, const float* d1, int D, int iters, const int* init, float* protos,
                             int* assign, char* ws, cudaStream_t st) {
    const KmLayout l = km_layout(g, D);
    float* A = reinterpret_cast<float*>(ws + l.A);
    unsigned long long* S = reinterpret_cast<unsigned long long*>(ws + l.S);
    unsigned int* cnt = reinterpret_cast<unsigned int*>(ws + l.cnt);
    const int P0 = g.P0x * g.P0y;
    const long long n = (long long)P0 * KD;
    const size_t smem = (size_t)KD * (ASTR + CSTR) * sizeof(float);
    static std::atomic<unsigned long long> smem_done{0};
    cudaError_t e = dm_smem_opt_in(reinterpret_cast<const void*>(k_km_assign), (int)smem, smem_done);
    if (e != cudaSuccess) return e;
    float* part_s = reinterpret_cast<float*>(ws + l.part_s);
    int* part_i = reinterpret_cast<int*>(ws + l.part_i);
    const unsigned nb = (unsigned)((n + 255) / 256);
    const dim3 ag((unsigned)((P0 + KM_BM - 1) / KM_BM), (unsigned)l.nchunk);
    const unsigned mb = (unsigned)((P0 + 255) / 256);
    k_patch_vectors<<<nb, 256, 0, st>>>(g, d1, A);
    k_km_init<<<D, 160, 0, st>>>(A, init, protos);
    long long launches = 2;
    for (int it = 0; it < iters; it++) {
        k_km_assign<<<ag, 256, smem, st>>>(A, P0, protos, D, l.chunk, part_s, part_i);
        k_km_merge<<<mb, 256, 0, st>>>(part_s, part_i, P0, l.nchunk, D, assign);
        if ((e = cudaMemsetAsync(S, 0, (size_t)D * KD * sizeof(unsigned long long), st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(cnt, 0, (size_t)D * sizeof(unsigned int), st)) != cudaSuccess) return e;
        k_km_accum<<<nb, 256, 0, st>>>(A, n, assign, S, cnt);
        k_km_finish<<<D, 160, 0, st>>>(S, cnt, protos);
        launches += 4;
    }
    k_km_assign<<<ag, 256, smem, st>>>(A, P0, protos, D, l.chunk, part_s, part_i);
    k_km_merge<<<mb, 256, 0, st>>>(part_s, part_i, P0, l.nchunk, D, assign);
    dm_count_launches(launches + 2);
    return cudaGetLastError();
}

// Offset of the D-int init array inside the k-means workspace (the API copies
// the caller's host indices there).
size_t dm_kmeans_init_offset(const DmGeom& g, int D) { return km_layout(g, D).init; }
