// Scale and rotation invariant form (Sec. 4.2, Algorithm 2): the transform
// list, the similarity warp of an image onto its canvas, and the fold of one
// transform's device status into the call's header.
//
// Algorithm 2 runs the matching on I downsized by sigma1 against I' downsized
// by sigma2 and rotated by -theta, for sigma = -2, -1.5, .., 2 and theta = k
// pi/4, and pools the rectified atomic correspondences of all 72 runs before
// one reciprocal verification.  The paper does not say how the images are
// resampled; here:
//   * the canvas is the bounding box of the scaled, rotated image (nothing is
//     cropped), its size rounded to the nearest integer in double precision;
//   * canvas pixel (u, v) samples the image bilinearly at
//     image centre + sigma R_theta ((u, v) - canvas centre), zero outside the
//     image, with no prefilter (the descriptors' own smoothing follows);
//   * the coordinates are computed in FP32 in the fixed order of dm_to_source,
//     the bilinear blend as top = p00 + fx (p10 - p00), bot = p01 + fx (p11 -
//     p01), top + fy (bot - top), each operation rounded once.
#include <math.h>

#include "dm_internal.cuh"

namespace {

// 2^(|sigma|) for |sigma| = 0, 0.5, .., 2 and cos / sin of k pi/4: the values
// nearest to the definitions in double precision.
constexpr double kScale[5] = {1.0, 1.4142135623730951, 2.0, 2.8284271247461903, 4.0};
constexpr double kHalfSqrt2 = 0.70710678118654752440;
constexpr double kCos[8] = {1.0, kHalfSqrt2, 0.0, -kHalfSqrt2, -1.0, -kHalfSqrt2, 0.0, kHalfSqrt2};
constexpr double kSin[8] = {0.0, kHalfSqrt2, 1.0, kHalfSqrt2, 0.0, -kHalfSqrt2, -1.0, -kHalfSqrt2};

// Canvas of a W x H image downsized by sigma and rotated by k pi/4.
void canvas(int W, int H, double sigma, int k, int* Wr, int* Hr) {
    const double c = fabs(kCos[k]), s = fabs(kSin[k]);
    const double w = floor(((double)W * c + (double)H * s) / sigma + 0.5);
    const double h = floor(((double)W * s + (double)H * c) / sigma + 0.5);
    *Wr = w < 1.0 ? 1 : (int)w;
    *Hr = h < 1.0 ? 1 : (int)h;
}

__global__ void k_warp(const float* __restrict__ img, int W, int H, float* __restrict__ out, int Wr, int Hr,
                       DmXform t) {
    const long long n = (long long)Wr * Hr;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int u = (int)(i % Wr), v = (int)(i / Wr);
        float x, y;
        dm_to_source(t, (float)u, (float)v, x, y);
        const float x0 = floorf(x), y0 = floorf(y);
        const float fx = __fsub_rn(x, x0), fy = __fsub_rn(y, y0);
        const int xi = (int)x0, yi = (int)y0;
        auto px = [&](int yy, int xx) -> float {
            return (xx >= 0 && yy >= 0 && xx < W && yy < H) ? __ldg(img + (size_t)yy * W + xx) : 0.0f;
        };
        const float p00 = px(yi, xi), p10 = px(yi, xi + 1), p01 = px(yi + 1, xi), p11 = px(yi + 1, xi + 1);
        const float top = __fadd_rn(p00, __fmul_rn(fx, __fsub_rn(p10, p00)));
        const float bot = __fadd_rn(p01, __fmul_rn(fx, __fsub_rn(p11, p01)));
        out[i] = __fadd_rn(top, __fmul_rn(fy, __fsub_rn(bot, top)));
    }
}

// Transforms may run on concurrent streams: every update of the call's header
// is atomic.  A count that wraps is set to the maximum (saturation).
__global__ void k_inv_fold(DmWsHeader* __restrict__ dst, const DmWsHeader* __restrict__ src) {
    const int i = threadIdx.x;
    if (i == 0) {
        if (src->status) atomicOr(&dst->status, src->status);
        if (src->pyr_status) atomicOr(&dst->pyr_status, src->pyr_status);
    }
    if (i < DM_MAXL + 2) {
        const unsigned int v = src->count[i];
        const unsigned int old = atomicAdd(&dst->count[i], v);
        if (old + v < old) atomicExch(&dst->count[i], 0xffffffffu);
    }
}

}  // namespace

void dm_invariant_transform(int i, int W1, int H1, int W2, int H2, DmInvTransform* t) {
    const int j = i / 8, a = j < 4 ? 4 - j : j - 4;
    t->k = i % 8;
    t->s1 = j >= 4 ? kScale[a] : 1.0;
    t->s2 = j < 4 ? kScale[a] : 1.0;
    canvas(W1, H1, t->s1, 0, &t->w1, &t->h1);
    canvas(W2, H2, t->s2, t->k, &t->w2, &t->h2);
}

DmXform dm_make_xform(int W, int H, int Wr, int Hr, double sigma, int k) {
    DmXform t;
    t.cu = (float)((Wr - 1) * 0.5);
    t.cv = (float)((Hr - 1) * 0.5);
    t.cx = (float)((W - 1) * 0.5);
    t.cy = (float)((H - 1) * 0.5);
    t.sg = (float)sigma;
    t.c = (float)kCos[k];
    t.s = (float)kSin[k];
    return t;
}

cudaError_t dm_launch_warp(const float* img, int W, int H, float* out, int Wr, int Hr, const DmXform& t,
                           cudaStream_t st) {
    const long long n = (long long)Wr * Hr;
    const long long nb = (n + 255) / 256;
    k_warp<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, st>>>(img, W, H, out, Wr, Hr, t);
    dm_count_launches(1);
    return cudaGetLastError();
}

cudaError_t dm_launch_inv_fold(DmWsHeader* dst, const DmWsHeader* src, cudaStream_t st) {
    k_inv_fold<<<1, 64, 0, st>>>(dst, src);
    dm_count_launches(1);
    return cudaGetLastError();
}
