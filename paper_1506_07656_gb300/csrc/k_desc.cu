// Pixel descriptors (Sec. 3.2 "Pixel descriptor").
//
// Pipeline per image: s = image_scale * I; Gaussian nu1 (horizontal pass,
// then vertical); central-difference gradient with replicated border;
// non-negative projections on the directions k*pi/4, k = 0..7; Gaussian nu2
// on each channel; sigmoid 2/(1+exp(-slope x)) - 1; Gaussian nu3; append mu
// and L2-normalise the 9-vector.  Every step is an elementwise or separable
// stencil pass over a few MB, so each is one simple kernel; the operation
// order inside each output is fixed (an fma chain over taps j = -R..R from 0)
// so the FP32 result is reproducible bit for bit.
#include "dm_internal.cuh"

#include <algorithm>
#include <cstring>

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Horizontal pass of one channel plane set.  in: [H][W][C] (C = 1 or 8);
// scale applied to the input value first when `scale_in` != 1 (first pass).
template <int C>
__device__ __forceinline__ void smooth_h(const float* __restrict__ in, float* __restrict__ out, int W, int H,
                                         const DmTaps& t, float scale_in, int apply_scale, long long idx) {
    long long n = (long long)W * H * C;
    if (idx >= n) return;
    int c = (int)(idx % C);
    long long pix = idx / C;
    int x = (int)(pix % W), y = (int)(pix / W);
    const float* row = in + (long long)y * W * C;
    float acc = 0.0f;
    for (int j = -t.R; j <= t.R; j++) {
        float v = row[(long long)clampi(x + j, 0, W - 1) * C + c];
        if (apply_scale) v = __fmul_rn(v, scale_in);
        acc = __fmaf_rn(t.w[j + t.R], v, acc);
    }
    out[idx] = acc;
}

// Vertical pass; post = 0 none, 1 sigmoid, 2 normalise into [H][W][9] output.
template <int C, int POST>
__device__ __forceinline__ void smooth_v(const float* __restrict__ in, float* __restrict__ out, int W, int H,
                                         const DmTaps& t, float slope, float mu, long long gidx) {
    if (POST == 2) {
        // one thread per pixel: smooth its C channels, then normalise
        long long pix = gidx;
        if (pix >= (long long)W * H) return;
        int x = (int)(pix % W), y = (int)(pix / W);
        float v[C];
#pragma unroll
        for (int c = 0; c < C; c++) {
            float acc = 0.0f;
            for (int j = -t.R; j <= t.R; j++)
                acc = __fmaf_rn(t.w[j + t.R], in[((long long)clampi(y + j, 0, H - 1) * W + x) * C + c], acc);
            v[c] = acc;
        }
        float acc = 0.0f;
#pragma unroll
        for (int c = 0; c < C; c++) acc = __fmaf_rn(v[c], v[c], acc);
        acc = __fmaf_rn(mu, mu, acc);
        float nrm = __fsqrt_rn(acc);
        float* o = out + pix * 9;
#pragma unroll
        for (int c = 0; c < C; c++) o[c] = __fdiv_rn(v[c], nrm);
        o[8] = __fdiv_rn(mu, nrm);
        return;
    }
    const long long idx = gidx;
    long long n = (long long)W * H * C;
    if (idx >= n) return;
    int c = (int)(idx % C);
    long long pix = idx / C;
    int x = (int)(pix % W), y = (int)(pix / W);
    float acc = 0.0f;
    for (int j = -t.R; j <= t.R; j++)
        acc = __fmaf_rn(t.w[j + t.R], in[((long long)clampi(y + j, 0, H - 1) * W + x) * C + c], acc);
    if (POST == 1) {
        float tt = __fmul_rn(slope, acc);
        float e = dm_expf(-tt);
        float d = __fadd_rn(1.0f, e);
        acc = __fsub_rn(__fdiv_rn(2.0f, d), 1.0f);
    }
    out[idx] = acc;
}

// Elementwise sigmoid (used when nu2 = 0, i.e. no vertical pass to fuse into).
__global__ void k_sigmoid(float* __restrict__ buf, long long n, float slope) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    float tt = __fmul_rn(slope, buf[idx]);
    float e = dm_expf(-tt);
    float d = __fadd_rn(1.0f, e);
    buf[idx] = __fsub_rn(__fdiv_rn(2.0f, d), 1.0f);
}

// Scale without smoothing (nu1 = 0).
__global__ void k_scale(const float* __restrict__ in, float* __restrict__ out, long long n, float s) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] = __fmul_rn(in[idx], s);
}

// Gradient + 8 non-negative projections.  dir_k = (cos k pi/4, sin k pi/4)
// with the exact table {1, r, 0, -r, -1, -r, 0, r} / {0, r, 1, r, 0, -r, -1, -r},
// r = sqrt(1/2) rounded to float; v_k = fma(gx, cos_k, gy * sin_k), then max(v, 0).
__device__ __forceinline__ void grad_proj(const float* __restrict__ s, float* __restrict__ o8, int W, int H, long long pix) {
    if (pix >= (long long)W * H) return;
    int x = (int)(pix % W), y = (int)(pix / W);
    float gx = __fmul_rn(__fsub_rn(s[(long long)y * W + clampi(x + 1, 0, W - 1)], s[(long long)y * W + clampi(x - 1, 0, W - 1)]), 0.5f);
    float gy = __fmul_rn(__fsub_rn(s[(long long)clampi(y + 1, 0, H - 1) * W + x], s[(long long)clampi(y - 1, 0, H - 1) * W + x]), 0.5f);
    const float r = 0.70710678118654752f;
    const float dc[8] = {1.0f, r, 0.0f, -r, -1.0f, -r, 0.0f, r};
    const float ds[8] = {0.0f, r, 1.0f, r, 0.0f, -r, -1.0f, -r};
    float* o = o8 + pix * 8;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        float v = __fmaf_rn(gx, dc[k], __fmul_rn(gy, ds[k]));
        o[k] = v > 0.0f ? v : 0.0f;
    }
}

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }

template <int C>
__global__ void k_smooth_h(const float* __restrict__ in, float* __restrict__ out, int W, int H, DmTaps t, float scale_in,
                           int apply_scale) {
    smooth_h<C>(in, out, W, H, t, scale_in, apply_scale, gtid());
}
template <int C, int POST>
__global__ void k_smooth_v(const float* __restrict__ in, float* __restrict__ out, int W, int H, DmTaps t, float slope,
                           float mu) {
    smooth_v<C, POST>(in, out, W, H, t, slope, mu, gtid());
}
__global__ void k_grad_proj(const float* __restrict__ s, float* __restrict__ o8, int W, int H) { grad_proj(s, o8, W, H, gtid()); }

// Cross-pair form: the same passes for every image of a wave of the batched
// form in one launch each, image blockIdx.y (its buffers in the parameters).
struct IoBatch {
    const float* in[2 * DM_BATCH_MAX];
    float* out[2 * DM_BATCH_MAX];
    int W[2 * DM_BATCH_MAX], H[2 * DM_BATCH_MAX];
    int n;
};
template <int C>
__global__ void k_smooth_h_b(const __grid_constant__ IoBatch B, DmTaps t, float scale_in, int apply_scale) {
    const int i = blockIdx.y;
    smooth_h<C>(B.in[i], B.out[i], B.W[i], B.H[i], t, scale_in, apply_scale, gtid());
}
template <int C, int POST>
__global__ void k_smooth_v_b(const __grid_constant__ IoBatch B, DmTaps t, float slope, float mu) {
    const int i = blockIdx.y;
    smooth_v<C, POST>(B.in[i], B.out[i], B.W[i], B.H[i], t, slope, mu, gtid());
}
__global__ void k_grad_proj_b(const __grid_constant__ IoBatch B) {
    const int i = blockIdx.y;
    grad_proj(B.in[i], B.out[i], B.W[i], B.H[i], gtid());
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// tmpA, tmpB: [H][W][8] float each.
cudaError_t dm_launch_descriptors(const DmDescParams& prm, const float* img, int W, int H, float* desc,
                                  float* tmpA, float* tmpB, cudaStream_t st) {
    const int B = 256;
    long long n1 = (long long)W * H, n8 = n1 * 8;
    // s = scale * I, smoothed by nu1 -> tmpB (1 channel)
    if (prm.t1.R > 0) {
        k_smooth_h<1><<<nblk(n1, B), B, 0, st>>>(img, tmpA, W, H, prm.t1, prm.scale, 1);
        k_smooth_v<1, 0><<<nblk(n1, B), B, 0, st>>>(tmpA, tmpB, W, H, prm.t1, 0.f, 0.f);
    } else {
        k_scale<<<nblk(n1, B), B, 0, st>>>(img, tmpB, n1, prm.scale);
    }
    // gradient projections -> tmpA [H][W][8]
    k_grad_proj<<<nblk(n1, B), B, 0, st>>>(tmpB, tmpA, W, H);
    // nu2 smoothing + sigmoid -> tmpA
    if (prm.t2.R > 0) {
        k_smooth_h<8><<<nblk(n8, B), B, 0, st>>>(tmpA, tmpB, W, H, prm.t2, 1.f, 0);
        k_smooth_v<8, 1><<<nblk(n8, B), B, 0, st>>>(tmpB, tmpA, W, H, prm.t2, prm.slope, 0.f);
    } else {
        k_sigmoid<<<nblk(n8, B), B, 0, st>>>(tmpA, n8, prm.slope);
    }
    // nu3 smoothing + normalisation -> desc [H][W][9]
    const float* src = tmpA;
    if (prm.t3.R > 0) {
        k_smooth_h<8><<<nblk(n8, B), B, 0, st>>>(tmpA, tmpB, W, H, prm.t3, 1.f, 0);
        src = tmpB;
    }
    DmTaps id;
    id.R = 0;
    id.w[0] = 1.0f;
    k_smooth_v<8, 2><<<nblk(n1, B), B, 0, st>>>(src, desc, W, H, prm.t3.R > 0 ? prm.t3 : id, 0.f, prm.mu);
    dm_count_launches((prm.t1.R > 0 ? 2 : 1) + 1 + (prm.t2.R > 0 ? 2 : 1) + (prm.t3.R > 0 ? 1 : 0) + 1);
    return cudaGetLastError();
}

// One image scaled by `scale` and smoothed by taps t (horizontal pass, then
// vertical), as the first step of the descriptors; R = 0: scaled only.
cudaError_t dm_launch_smooth1(const float* img, int W, int H, float scale, const DmTaps& t, float* out, float* tmp,
                              cudaStream_t st) {
    const int B = 256;
    const long long n1 = (long long)W * H;
    if (t.R > 0) {
        k_smooth_h<1><<<nblk(n1, B), B, 0, st>>>(img, tmp, W, H, t, scale, 1);
        k_smooth_v<1, 0><<<nblk(n1, B), B, 0, st>>>(tmp, out, W, H, t, 0.f, 0.f);
        dm_count_launches(2);
    } else {
        k_scale<<<nblk(n1, B), B, 0, st>>>(img, out, n1, scale);
        dm_count_launches(1);
    }
    return cudaGetLastError();
}

// Descriptors of n <= 2 DM_BATCH_MAX images (a wave of the batched form): one
// launch per pass for all of them.  (With a zero smoothing width the scaling
// and sigmoid passes run image by image.)
cudaError_t dm_launch_descriptors_batch(const DmDescParams& prm, int n, const float* const* imgs, const int* Ws,
                                        const int* Hs, float* const* descs, float* const* tmpAs, float* const* tmpBs,
                                        cudaStream_t st) {
    if (n < 1 || n > 2 * DM_BATCH_MAX) return cudaErrorInvalidValue;
    if (prm.t1.R == 0 || prm.t2.R == 0 || prm.t3.R == 0) {
        for (int i = 0; i < n; i++) {
            cudaError_t e = dm_launch_descriptors(prm, imgs[i], Ws[i], Hs[i], descs[i], tmpAs[i], tmpBs[i], st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    const int B = 256;
    long long n1 = 0;
    for (int i = 0; i < n; i++) n1 = std::max(n1, (long long)Ws[i] * Hs[i]);
    const long long n8 = 8 * n1;
    auto io = [&](int step) {
        IoBatch b;
        memset(&b, 0, sizeof(b));
        b.n = n;
        for (int i = 0; i < n; i++) {
            b.W[i] = Ws[i];
            b.H[i] = Hs[i];
            switch (step) {
                case 0: b.in[i] = imgs[i]; b.out[i] = tmpAs[i]; break;     // nu1, horizontal
                case 1: b.in[i] = tmpAs[i]; b.out[i] = tmpBs[i]; break;    // nu1, vertical
                case 2: b.in[i] = tmpBs[i]; b.out[i] = tmpAs[i]; break;    // gradient projections
                case 3: b.in[i] = tmpAs[i]; b.out[i] = tmpBs[i]; break;    // nu2, horizontal
                case 4: b.in[i] = tmpBs[i]; b.out[i] = tmpAs[i]; break;    // nu2, vertical + sigmoid
                case 5: b.in[i] = tmpAs[i]; b.out[i] = tmpBs[i]; break;    // nu3, horizontal
                default: b.in[i] = tmpBs[i]; b.out[i] = descs[i]; break;   // nu3, vertical + normalisation
            }
        }
        return b;
    };
    const dim3 g1(nblk(n1, B), (unsigned)n), g8(nblk(n8, B), (unsigned)n);
    k_smooth_h_b<1><<<g1, B, 0, st>>>(io(0), prm.t1, prm.scale, 1);
    k_smooth_v_b<1, 0><<<g1, B, 0, st>>>(io(1), prm.t1, 0.f, 0.f);
    k_grad_proj_b<<<g1, B, 0, st>>>(io(2));
    k_smooth_h_b<8><<<g8, B, 0, st>>>(io(3), prm.t2, 1.f, 0);
    k_smooth_v_b<8, 1><<<g8, B, 0, st>>>(io(4), prm.t2, prm.slope, 0.f);
    k_smooth_h_b<8><<<g8, B, 0, st>>>(io(5), prm.t3, 1.f, 0);
    k_smooth_v_b<8, 2><<<g1, B, 0, st>>>(io(6), prm.t3, 0.f, prm.mu);
    dm_count_launches(7);
    return cudaGetLastError();
}
