// DeepFlow (Sec. 4.3): variational refinement of a flow field with the
// DeepMatching matches as one of its terms.
//
// Energy E = int delta Psi(theta0 (grad3 I . w)^2) + gamma Psi(normalised
// gradient constancy) + alpha(x) Psi(|grad u|^2 + |grad v|^2) + beta_k c phi
// Psi(|w - w'|^2), Psi(s^2) = sqrt(s^2 + eps^2), minimised coarse to fine
// (factor eta) with warping; per level n_fixed fixed-point steps (the robust
// weights recomputed from the current increment), each solved approximately
// by n_sor red-black SOR sweeps.  Every step is a data-parallel pass over the
// pixels of one level; the arithmetic is FP32 with one fixed order of
// correctly rounded operations, the same as the FP32 reference.  The
// choices the paper leaves open (resampling, stencils, border rules, where a
// match lands on a coarse level, SOR ordering) are stated at each kernel.
//
// Levels whose pixels fit one CTA's sweep (small levels, most of the 60-odd
// levels of a VGA-sized pair) run all their fixed-point steps and SOR sweeps
// in one kernel with block barriers between sweeps; larger levels launch one
// kernel per step and colour.
#include <math.h>

#include "dm_internal.cuh"

namespace {

struct DfConst {
    float scale, kappa, gamma, delta, zeta2, eps2, omega, one_m_omega, sigma_m, two_sigma_m, norm;
};

__device__ __forceinline__ float df_at(const float* f, int W, int x, int y) { return f[(size_t)y * W + x]; }

// Central differences with a replicated border.
__device__ __forceinline__ float df_dx(const float* f, int W, int x, int y) {
    return __fmul_rn(0.5f, __fsub_rn(df_at(f, W, x + 1 < W ? x + 1 : W - 1, y), df_at(f, W, x > 0 ? x - 1 : 0, y)));
}
__device__ __forceinline__ float df_dy(const float* f, int W, int H, int x, int y) {
    return __fmul_rn(0.5f, __fsub_rn(df_at(f, W, x, y + 1 < H ? y + 1 : H - 1), df_at(f, W, x, y > 0 ? y - 1 : 0)));
}

// Bilinear sample at (xs, ys), coordinates clamped to the image.
__device__ __forceinline__ float df_bilinear(const float* f, int W, int H, float xs, float ys) {
    xs = xs < 0.0f ? 0.0f : xs;
    ys = ys < 0.0f ? 0.0f : ys;
    xs = xs > (float)(W - 1) ? (float)(W - 1) : xs;
    ys = ys > (float)(H - 1) ? (float)(H - 1) : ys;
    const float fx0 = floorf(xs), fy0 = floorf(ys);
    const int x0 = (int)fx0, y0 = (int)fy0;
    const int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    const float fx = __fsub_rn(xs, fx0), fy = __fsub_rn(ys, fy0);
    const float p00 = df_at(f, W, x0, y0), p10 = df_at(f, W, x1, y0), p01 = df_at(f, W, x0, y1), p11 = df_at(f, W, x1, y1);
    const float top = __fadd_rn(p00, __fmul_rn(fx, __fsub_rn(p10, p00)));
    const float bot = __fadd_rn(p01, __fmul_rn(fx, __fsub_rn(p11, p01)));
    return __fadd_rn(top, __fmul_rn(fy, __fsub_rn(bot, top)));
}

// Psi'(s2) = 1 / (2 sqrt(s2 + eps^2)).
__device__ __forceinline__ float df_dpsi(float s2, float eps2) { return __fdiv_rn(0.5f, __fsqrt_rn(__fadd_rn(s2, eps2))); }

// Level resampling: dst pixel x samples src at (x + 1/2) / s - 1/2 (down,
// s = eta: the next coarser level) or (x + 1/2) s - 1/2 (up, s = eta: the
// flow carried to the finer level), times mul.
__global__ void k_df_resample(const float* __restrict__ src, int Ws, int Hs, float* __restrict__ dst, int Wd, int Hd,
                              float s, int down, float mul) {
    const long long n = (long long)Wd * Hd;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Wd), y = (int)(i / Wd);
        const float cx = __fadd_rn((float)x, 0.5f), cy = __fadd_rn((float)y, 0.5f);
        const float xs = down ? __fsub_rn(__fdiv_rn(cx, s), 0.5f) : __fsub_rn(__fmul_rn(cx, s), 0.5f);
        const float ys = down ? __fsub_rn(__fdiv_rn(cy, s), 0.5f) : __fsub_rn(__fmul_rn(cy, s), 0.5f);
        dst[i] = __fmul_rn(df_bilinear(src, Ws, Hs, xs, ys), mul);
    }
}

__device__ __forceinline__ int df_clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int df_count(const int* d_count, int capacity) {
    const int n = *d_count;
    return n < 0 ? 0 : (n > capacity ? capacity : n);
}

// Weight phi of each match at full resolution: lambda~ = 10 x the smaller
// eigenvalue of the 3x3 sum of gradient products of I1 around x1; Delta =
// |I1(x1) - I2(x2)| + |dx I1(x1) - dx I2(x2)| + |dy I1(x1) - dy I2(x2)|;
// phi = sqrt(lambda~) / (sigma_M sqrt(2 pi)) exp(-Delta / (2 sigma_M)).
__global__ void k_df_phi(const float* __restrict__ I1, const float* __restrict__ I2, int W, int H,
                         const dm_match_t* __restrict__ m, const int* __restrict__ d_count, int capacity, DfConst k,
                         float* __restrict__ phi) {
    const int n = df_count(d_count, capacity);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int x1 = df_clampi((int)m[i].x1, 0, W - 1), y1 = df_clampi((int)m[i].y1, 0, H - 1);
        const int x2 = df_clampi((int)m[i].x2, 0, W - 1), y2 = df_clampi((int)m[i].y2, 0, H - 1);
        float a = 0.0f, b = 0.0f, c = 0.0f;
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                const int xx = df_clampi(x1 + dx, 0, W - 1), yy = df_clampi(y1 + dy, 0, H - 1);
                const float gx = df_dx(I1, W, xx, yy), gy = df_dy(I1, W, H, xx, yy);
                a = __fadd_rn(a, __fmul_rn(gx, gx));
                b = __fadd_rn(b, __fmul_rn(gx, gy));
                c = __fadd_rn(c, __fmul_rn(gy, gy));
            }
        const float h = __fmul_rn(__fsub_rn(a, c), 0.5f);
        float lmin = __fsub_rn(__fmul_rn(__fadd_rn(a, c), 0.5f), __fsqrt_rn(__fadd_rn(__fmul_rn(h, h), __fmul_rn(b, b))));
        if (lmin < 0.0f) lmin = 0.0f;
        const float lt = __fmul_rn(10.0f, lmin);
        float d = fabsf(__fsub_rn(df_at(I1, W, x1, y1), df_at(I2, W, x2, y2)));
        d = __fadd_rn(d, fabsf(__fsub_rn(df_dx(I1, W, x1, y1), df_dx(I2, W, x2, y2))));
        d = __fadd_rn(d, fabsf(__fsub_rn(df_dy(I1, W, H, x1, y1), df_dy(I2, W, H, x2, y2))));
        const float z = -__fdiv_rn(d, k.two_sigma_m);
        phi[i] = __fmul_rn(__fmul_rn(__fdiv_rn(__fsqrt_rn(lt), k.sigma_m), k.norm), dm_expf(z));
    }
}

// Matches on level k: match i lands on pixel round((x1 + 1/2) s_k - 1/2)
// (clamped); a pixel keeps the match with the higher DeepMatching score, then
// the lower index (64-bit key: order-preserving score bits, then ~index).
__device__ __forceinline__ unsigned int df_score_key(float s) {
    const unsigned int b = __float_as_uint(s);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void k_df_raster(const dm_match_t* __restrict__ m, const int* __restrict__ d_count, int capacity, int w, int h,
                            float sk, unsigned long long* __restrict__ owner) {
    const int n = df_count(d_count, capacity);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float fx = __fsub_rn(__fmul_rn(__fadd_rn(m[i].x1, 0.5f), sk), 0.5f);
        const float fy = __fsub_rn(__fmul_rn(__fadd_rn(m[i].y1, 0.5f), sk), 0.5f);
        const int px = df_clampi((int)floorf(__fadd_rn(fx, 0.5f)), 0, w - 1);
        const int py = df_clampi((int)floorf(__fadd_rn(fy, 0.5f)), 0, h - 1);
        const unsigned long long key = ((unsigned long long)df_score_key(m[i].score) << 32) | (0xffffffffu - (unsigned int)i);
        atomicMax(owner + (size_t)py * w + px, key);
    }
}

// Per pixel: beta_k phi, u', v' of the winning match (0 where none).
__global__ void k_df_match_fields(const unsigned long long* __restrict__ owner, const dm_match_t* __restrict__ m,
                                  const float* __restrict__ phi, int n_px, float beta_k, float sk, float* __restrict__ mc,
                                  float* __restrict__ mu, float* __restrict__ mv) {
    for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n_px; o += gridDim.x * blockDim.x) {
        const unsigned long long key = owner[o];
        float c = 0.0f, a = 0.0f, b = 0.0f;
        if (key != 0ull) {
            const int i = (int)(0xffffffffu - (unsigned int)key);
            c = __fmul_rn(beta_k, phi[i]);
            a = __fmul_rn(__fsub_rn(m[i].x2, m[i].x1), sk);
            b = __fmul_rn(__fsub_rn(m[i].y2, m[i].y1), sk);
        }
        mc[o] = c;
        mu[o] = a;
        mv[o] = b;
    }
}

// Linearisation around the current flow, step 1: alpha(x) = exp(-kappa
// |grad I1| / 255), the warped I2w = I2(x + w) (bilinear, clamped) and the
// mean Im = (I1 + I2w) / 2.
__global__ void k_df_prep1(const float* __restrict__ I1, const float* __restrict__ I2, const float* __restrict__ u,
                           const float* __restrict__ v, int w, int h, DfConst k, float* __restrict__ alpha,
                           float* __restrict__ I2w, float* __restrict__ Im) {
    const long long n = (long long)w * h;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % w), y = (int)(o / w);
        const float gx = __fdiv_rn(df_dx(I1, w, x, y), k.scale), gy = __fdiv_rn(df_dy(I1, w, h, x, y), k.scale);
        alpha[o] = dm_expf(-__fmul_rn(k.kappa, __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)))));
        const float wv = df_bilinear(I2, w, h, __fadd_rn((float)x, u[o]), __fadd_rn((float)y, v[o]));
        I2w[o] = wv;
        Im[o] = __fmul_rn(0.5f, __fadd_rn(I1[o], wv));
    }
}

// Step 2: first derivatives of the mean image.
__global__ void k_df_prep2(const float* __restrict__ Im, int w, int h, float* __restrict__ Ix, float* __restrict__ Iy) {
    const long long n = (long long)w * h;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % w), y = (int)(o / w);
        Ix[o] = df_dx(Im, w, x, y);
        Iy[o] = df_dy(Im, w, h, x, y);
    }
}

// Step 3: the 11 per-pixel data-term quantities D = (Ix, Iy, Iz, Ixx, Ixy,
// Iyy, Ixz, Iyz, theta0, thetax, thetay), structure-of-arrays with stride n:
// Iz = I2w - I1; Ixx = dx(Ix), Ixy = dy(Ix), Iyy = dy(Iy); Ixz = dx(I2w) -
// dx(I1), Iyz = dy(I2w) - dy(I1); theta0 = 1 / (Ix^2 + Iy^2 + zeta^2),
// thetax = 1 / (Ixx^2 + Ixy^2 + zeta^2), thetay = 1 / (Ixy^2 + Iyy^2 + zeta^2).
__global__ void k_df_prep3(const float* __restrict__ I1, const float* __restrict__ I2w, const float* __restrict__ Ixa,
                           const float* __restrict__ Iya, int w, int h, DfConst k, float* __restrict__ D) {
    const long long n = (long long)w * h;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(o % w), y = (int)(o / w);
        const float Ix = Ixa[o], Iy = Iya[o];
        const float Ixx = df_dx(Ixa, w, x, y), Ixy = df_dy(Ixa, w, h, x, y), Iyy = df_dy(Iya, w, h, x, y);
        D[o] = Ix;
        D[n + o] = Iy;
        D[2 * n + o] = __fsub_rn(I2w[o], I1[o]);
        D[3 * n + o] = Ixx;
        D[4 * n + o] = Ixy;
        D[5 * n + o] = Iyy;
        D[6 * n + o] = __fsub_rn(df_dx(I2w, w, x, y), df_dx(I1, w, x, y));
        D[7 * n + o] = __fsub_rn(df_dy(I2w, w, h, x, y), df_dy(I1, w, h, x, y));
        D[8 * n + o] = __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(__fmul_rn(Ix, Ix), __fmul_rn(Iy, Iy)), k.zeta2));
        D[9 * n + o] = __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(__fmul_rn(Ixx, Ixx), __fmul_rn(Ixy, Ixy)), k.zeta2));
        D[10 * n + o] = __fdiv_rn(1.0f, __fadd_rn(__fadd_rn(__fmul_rn(Ixy, Ixy), __fmul_rn(Iyy, Iyy)), k.zeta2));
    }
}

// Fixed-point step, per pixel o: the smoothness weight psi_s = alpha
// Psi'(|grad(u + du)|^2 + |grad(v + dv)|^2) from forward differences (0 at the
// last column / row), the robust data and matching weights at the current
// increment, and the 2x2 system A = (A11, A12, A22, b1, b2) (structure of
// arrays, stride n).
struct DfLevel {
    int w, h;
    long long n;
    const float* D;        // [11][n]
    const float* alpha;
    const float* mc;       // beta_k phi at matched pixels, else 0
    const float* mu;
    const float* mv;
    const float* u;
    const float* v;
    float* du;
    float* dv;
    float* A;              // [5][n]
    float* ps;
};

__device__ __forceinline__ void df_weights_at(const DfLevel& L, const DfConst& k, long long o) {
    const int x = (int)(o % L.w), y = (int)(o / L.w);
    const long long n = L.n;
    const float* D = L.D;
    const float du = L.du[o], dv = L.dv[o];
    const float U = __fadd_rn(L.u[o], du), V = __fadd_rn(L.v[o], dv);
    float ux = 0.0f, uy = 0.0f, vx = 0.0f, vy = 0.0f;
    if (x + 1 < L.w) {
        ux = __fsub_rn(__fadd_rn(L.u[o + 1], L.du[o + 1]), U);
        vx = __fsub_rn(__fadd_rn(L.v[o + 1], L.dv[o + 1]), V);
    }
    if (y + 1 < L.h) {
        uy = __fsub_rn(__fadd_rn(L.u[o + L.w], L.du[o + L.w]), U);
        vy = __fsub_rn(__fadd_rn(L.v[o + L.w], L.dv[o + L.w]), V);
    }
    const float s2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(vx, vx)), __fmul_rn(vy, vy));
    L.ps[o] = __fmul_rn(L.alpha[o], df_dpsi(s2, k.eps2));
    const float d0 = D[o], d1 = D[n + o], d2 = D[2 * n + o], d3 = D[3 * n + o], d4 = D[4 * n + o], d5 = D[5 * n + o];
    const float d6 = D[6 * n + o], d7 = D[7 * n + o], d8 = D[8 * n + o], d9 = D[9 * n + o], d10 = D[10 * n + o];
    float a0 = 0.0f;
    if (k.delta > 0.0f) {
        const float r0 = __fadd_rn(__fadd_rn(__fmul_rn(d0, du), __fmul_rn(d1, dv)), d2);
        a0 = __fmul_rn(__fmul_rn(k.delta, df_dpsi(__fmul_rn(d8, __fmul_rn(r0, r0)), k.eps2)), d8);
    }
    const float rx = __fadd_rn(__fadd_rn(__fmul_rn(d3, du), __fmul_rn(d4, dv)), d6);
    const float ry = __fadd_rn(__fadd_rn(__fmul_rn(d4, du), __fmul_rn(d5, dv)), d7);
    const float ag = __fmul_rn(k.gamma, df_dpsi(__fadd_rn(__fmul_rn(d9, __fmul_rn(rx, rx)), __fmul_rn(d10, __fmul_rn(ry, ry))), k.eps2));
    float mw = 0.0f;
    const float mc = L.mc[o], mu = L.mu[o], mv = L.mv[o];
    if (mc > 0.0f) {
        const float eu = __fsub_rn(U, mu), ev = __fsub_rn(V, mv);
        mw = __fmul_rn(mc, df_dpsi(__fadd_rn(__fmul_rn(eu, eu), __fmul_rn(ev, ev)), k.eps2));
    }
    const float gx = __fmul_rn(ag, d9), gy = __fmul_rn(ag, d10);
    const float a0x = __fmul_rn(a0, d0), a0y = __fmul_rn(a0, d1);
    float* A = L.A;
    A[o] = __fadd_rn(__fadd_rn(__fmul_rn(a0x, d0), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d3), __fmul_rn(__fmul_rn(gy, d4), d4))), mw);
    A[n + o] = __fadd_rn(__fmul_rn(a0x, d1), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d4), __fmul_rn(__fmul_rn(gy, d4), d5)));
    A[2 * n + o] = __fadd_rn(__fadd_rn(__fmul_rn(a0y, d1), __fadd_rn(__fmul_rn(__fmul_rn(gx, d4), d4), __fmul_rn(__fmul_rn(gy, d5), d5))), mw);
    A[3 * n + o] = __fsub_rn(-__fadd_rn(__fmul_rn(a0x, d2), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d6), __fmul_rn(__fmul_rn(gy, d4), d7))),
                             __fmul_rn(mw, __fsub_rn(L.u[o], mu)));
    A[4 * n + o] = __fsub_rn(-__fadd_rn(__fmul_rn(a0y, d2), __fadd_rn(__fmul_rn(__fmul_rn(gx, d4), d6), __fmul_rn(__fmul_rn(gy, d5), d7))),
                             __fmul_rn(mw, __fsub_rn(L.v[o], mv)));
}

// One SOR relaxation of pixel o (red-black: its 4-neighbours have the other
// colour, so the pixels of one colour are independent): neighbours in the
// order left, right, up, down, edge weight (ps_o + ps_p) / 2;
//   du = (1 - omega) du + omega (b1 + sum w (du_p + u_p - u_o) - A12 dv) / (A11 + sum w),
// then dv the same way with the new du.
__device__ __forceinline__ void df_sor_at(const DfLevel& L, const DfConst& k, long long o) {
    const int x = (int)(o % L.w), y = (int)(o / L.w);
    const long long n = L.n;
    const float pso = L.ps[o], uo = L.u[o], vo = L.v[o];
    float sw = 0.0f, su = 0.0f, sv = 0.0f;
    long long nb[4];
    int nn = 0;
    if (x > 0) nb[nn++] = o - 1;
    if (x + 1 < L.w) nb[nn++] = o + 1;
    if (y > 0) nb[nn++] = o - L.w;
    if (y + 1 < L.h) nb[nn++] = o + L.w;
    for (int j = 0; j < nn; j++) {
        const long long p = nb[j];
        const float we = __fmul_rn(0.5f, __fadd_rn(pso, L.ps[p]));
        sw = __fadd_rn(sw, we);
        su = __fadd_rn(su, __fmul_rn(we, __fsub_rn(__fadd_rn(L.du[p], L.u[p]), uo)));
        sv = __fadd_rn(sv, __fmul_rn(we, __fsub_rn(__fadd_rn(L.dv[p], L.v[p]), vo)));
    }
    const float* A = L.A;
    const float a12 = A[n + o];
    const float nu = __fsub_rn(__fadd_rn(A[3 * n + o], su), __fmul_rn(a12, L.dv[o]));
    const float du = __fadd_rn(__fmul_rn(k.one_m_omega, L.du[o]), __fmul_rn(k.omega, __fdiv_rn(nu, __fadd_rn(A[o], sw))));
    L.du[o] = du;
    const float nv = __fsub_rn(__fadd_rn(A[4 * n + o], sv), __fmul_rn(a12, du));
    L.dv[o] = __fadd_rn(__fmul_rn(k.one_m_omega, L.dv[o]), __fmul_rn(k.omega, __fdiv_rn(nv, __fadd_rn(A[2 * n + o], sw))));
}

__global__ void k_df_weights(DfLevel L, DfConst k) {
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < L.n; o += (long long)gridDim.x * blockDim.x)
        df_weights_at(L, k, o);
}

// Pixels of one colour ((x + y) & 1 == color), indexed densely: row y holds
// ceil((w - start) / 2) of them, start = (y + color) & 1.
__global__ void k_df_sor(DfLevel L, DfConst k, int color) {
    const int half = (L.w + 1) / 2;
    const long long n = (long long)half * L.h;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(i / half), j = (int)(i % half);
        const int x = 2 * j + ((y + color) & 1);
        if (x < L.w) df_sor_at(L, k, (long long)y * L.w + x);
    }
}

__global__ void k_df_update(float* __restrict__ u, float* __restrict__ v, const float* __restrict__ du,
                            const float* __restrict__ dv, long long n) {
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        u[o] = __fadd_rn(u[o], du[o]);
        v[o] = __fadd_rn(v[o], dv[o]);
    }
}

// A whole small level in one CTA: n_fixed x (weights, then n_sor red-black
// sweeps), block barriers between the passes, then w += dw.  The same
// per-pixel operations as the multi-launch path.
constexpr int DF_SMALL_THREADS = 1024;

__global__ void __launch_bounds__(DF_SMALL_THREADS) k_df_level_small(DfLevel L, DfConst k, int n_fixed, int n_sor) {
    const int half = (L.w + 1) / 2;
    const long long nc = (long long)half * L.h;
    for (int it = 0; it < n_fixed; it++) {
        for (long long o = threadIdx.x; o < L.n; o += blockDim.x) df_weights_at(L, k, o);
        __syncthreads();
        for (int s = 0; s < n_sor; s++)
            for (int color = 0; color < 2; color++) {
                for (long long i = threadIdx.x; i < nc; i += blockDim.x) {
                    const int y = (int)(i / half), j = (int)(i % half);
                    const int x = 2 * j + ((y + color) & 1);
                    if (x < L.w) df_sor_at(L, k, (long long)y * L.w + x);
                }
                __syncthreads();
            }
    }
    float* u = const_cast<float*>(L.u);
    float* v = const_cast<float*>(L.v);
    for (long long o = threadIdx.x; o < L.n; o += blockDim.x) {
        u[o] = __fadd_rn(u[o], L.du[o]);
        v[o] = __fadd_rn(v[o], L.dv[o]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: the plan (level sizes, constants, workspace) and the launches.
// ---------------------------------------------------------------------------
namespace {
constexpr double kPi = 3.14159265358979323846;
constexpr long long DF_SMALL_MAX = 65536;      // pixels of a level solved by one CTA
inline unsigned df_blocks(long long n) {
    const long long b = (n + 255) / 256;
    return (unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}
}  // namespace

void dm_flow_plan(int W, int H, int capacity, const dm_flow_params& p, DmFlowPlan* q) {
    memset(q, 0, sizeof(*q));
    q->ws[0] = W;
    q->hs[0] = H;
    int n = 1;
    while (n < DM_DF_MAXLEVELS) {
        const int w = (int)floor(p.eta * q->ws[n - 1] + 0.5), h = (int)floor(p.eta * q->hs[n - 1] + 0.5);
        if (w < p.min_size || h < p.min_size) break;
        q->ws[n] = w;
        q->hs[n] = h;
        n++;
    }
    q->nl = n;
    const int kmax = n - 1;
    for (int k = 0; k < n; k++) {
        q->beta_k[k] = (float)(kmax > 0 ? p.beta * pow((double)k / (double)kmax, p.b) : p.beta);
        q->sk[k] = (float)pow(p.eta, (double)k);
    }
    q->eta = (float)p.eta;
    q->inv_eta = 1.0f / q->eta;
    q->scale = (float)p.image_scale;
    q->kappa = (float)p.kappa;
    q->gamma = (float)p.gamma;
    q->delta = (float)p.delta;
    q->zeta2 = (float)(p.zeta * p.zeta);
    q->eps2 = (float)(p.eps * p.eps);
    q->omega = (float)p.omega;
    q->one_m_omega = 1.0f - q->omega;
    q->sigma_m = (float)p.sigma_m;
    q->two_sigma_m = 2.0f * q->sigma_m;
    q->norm = (float)(1.0 / sqrt(2.0 * kPi));
    q->n_fixed = p.n_fixed;
    q->n_sor = p.n_sor;
    q->capacity = capacity;
    // workspace (floats unless stated): both pyramids, flow ping-pong, per-level scratch
    const size_t N0 = (size_t)W * H;
    size_t off = 0;
    for (int k = 0; k < n; k++) {
        const size_t Nk = (size_t)q->ws[k] * q->hs[k];
        q->P1[k] = off; off = dm_align(off + Nk * 4);
        q->P2[k] = off; off = dm_align(off + Nk * 4);
    }
    size_t* one[] = {&q->tmp, &q->fa_u, &q->fa_v, &q->fb_u, &q->fb_v, &q->du, &q->dv, &q->alpha, &q->I2w, &q->Im,
                     &q->Ix, &q->Iy, &q->ps, &q->mc, &q->mu, &q->mv};
    for (size_t* f : one) { *f = off; off = dm_align(off + N0 * 4); }
    q->D = off; off = dm_align(off + N0 * 11 * 4);
    q->A = off; off = dm_align(off + N0 * 5 * 4);
    q->owner = off; off = dm_align(off + N0 * 8);
    q->phi = off; off = dm_align(off + (size_t)(capacity > 0 ? capacity : 1) * 4);
    q->bytes = off;
}

cudaError_t dm_launch_deepflow(const DmFlowPlan& q, const DmTaps& taps, const float* img1, const float* img2,
                               const dm_match_t* m, const int* d_count, float* out_u, float* out_v, char* ws,
                               cudaStream_t st) {
    auto F = [&](size_t off) { return reinterpret_cast<float*>(ws + off); };
    DfConst k;
    k.scale = q.scale; k.kappa = q.kappa; k.gamma = q.gamma; k.delta = q.delta; k.zeta2 = q.zeta2; k.eps2 = q.eps2;
    k.omega = q.omega; k.one_m_omega = q.one_m_omega; k.sigma_m = q.sigma_m; k.two_sigma_m = q.two_sigma_m;
    k.norm = q.norm;
    const int W = q.ws[0], H = q.hs[0];
    long long launches = 0;
    cudaError_t e;
    if ((e = dm_launch_smooth1(img1, W, H, q.scale, taps, F(q.P1[0]), F(q.tmp), st)) != cudaSuccess) return e;
    if ((e = dm_launch_smooth1(img2, W, H, q.scale, taps, F(q.P2[0]), F(q.tmp), st)) != cudaSuccess) return e;
    for (int l = 1; l < q.nl; l++) {
        const long long n = (long long)q.ws[l] * q.hs[l];
        k_df_resample<<<df_blocks(n), 256, 0, st>>>(F(q.P1[l - 1]), q.ws[l - 1], q.hs[l - 1], F(q.P1[l]), q.ws[l], q.hs[l],
                                                    q.eta, 1, 1.0f);
        k_df_resample<<<df_blocks(n), 256, 0, st>>>(F(q.P2[l - 1]), q.ws[l - 1], q.hs[l - 1], F(q.P2[l]), q.ws[l], q.hs[l],
                                                    q.eta, 1, 1.0f);
        launches += 2;
    }
    const bool has_m = m != nullptr && d_count != nullptr && q.capacity > 0;
    if (has_m) {
        k_df_phi<<<df_blocks(q.capacity), 256, 0, st>>>(F(q.P1[0]), F(q.P2[0]), W, H, m, d_count, q.capacity, k, F(q.phi));
        launches++;
    }
    float* cu = F(q.fa_u);
    float* cv = F(q.fa_v);
    float* nu = F(q.fb_u);
    float* nv = F(q.fb_v);
    for (int l = q.nl - 1; l >= 0; l--) {
        const int w = q.ws[l], h = q.hs[l];
        const long long n = (long long)w * h;
        if (l == q.nl - 1) {
            if ((e = cudaMemsetAsync(cu, 0, n * 4, st)) != cudaSuccess) return e;
            if ((e = cudaMemsetAsync(cv, 0, n * 4, st)) != cudaSuccess) return e;
        } else {
            k_df_resample<<<df_blocks(n), 256, 0, st>>>(cu, q.ws[l + 1], q.hs[l + 1], nu, w, h, q.eta, 0, q.inv_eta);
            k_df_resample<<<df_blocks(n), 256, 0, st>>>(cv, q.ws[l + 1], q.hs[l + 1], nv, w, h, q.eta, 0, q.inv_eta);
            launches += 2;
            float* t = cu; cu = nu; nu = t;
            t = cv; cv = nv; nv = t;
        }
        // matches on this level
        if ((e = cudaMemsetAsync(ws + q.owner, 0, n * 8, st)) != cudaSuccess) return e;
        unsigned long long* owner = reinterpret_cast<unsigned long long*>(ws + q.owner);
        if (has_m) {
            k_df_raster<<<df_blocks(q.capacity), 256, 0, st>>>(m, d_count, q.capacity, w, h, q.sk[l], owner);
            launches++;
        }
        k_df_match_fields<<<df_blocks(n), 256, 0, st>>>(owner, m, F(q.phi), (int)n, q.beta_k[l], q.sk[l], F(q.mc), F(q.mu),
                                                         F(q.mv));
        // linearisation around the current flow
        k_df_prep1<<<df_blocks(n), 256, 0, st>>>(F(q.P1[l]), F(q.P2[l]), cu, cv, w, h, k, F(q.alpha), F(q.I2w), F(q.Im));
        k_df_prep2<<<df_blocks(n), 256, 0, st>>>(F(q.Im), w, h, F(q.Ix), F(q.Iy));
        k_df_prep3<<<df_blocks(n), 256, 0, st>>>(F(q.P1[l]), F(q.I2w), F(q.Ix), F(q.Iy), w, h, k, F(q.D));
        launches += 4;
        if ((e = cudaMemsetAsync(F(q.du), 0, n * 4, st)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(F(q.dv), 0, n * 4, st)) != cudaSuccess) return e;
        DfLevel L;
        L.w = w; L.h = h; L.n = n;
        L.D = F(q.D); L.alpha = F(q.alpha); L.mc = F(q.mc); L.mu = F(q.mu); L.mv = F(q.mv);
        L.u = cu; L.v = cv; L.du = F(q.du); L.dv = F(q.dv); L.A = F(q.A); L.ps = F(q.ps);
        if (n <= DF_SMALL_MAX) {
            k_df_level_small<<<1, DF_SMALL_THREADS, 0, st>>>(L, k, q.n_fixed, q.n_sor);
            launches++;
        } else {
            const long long nc = (long long)((w + 1) / 2) * h;
            for (int it = 0; it < q.n_fixed; it++) {
                k_df_weights<<<df_blocks(n), 256, 0, st>>>(L, k);
                for (int s = 0; s < q.n_sor; s++) {
                    k_df_sor<<<df_blocks(nc), 256, 0, st>>>(L, k, 0);
                    k_df_sor<<<df_blocks(nc), 256, 0, st>>>(L, k, 1);
                }
                launches += 1 + 2LL * q.n_sor;
            }
            k_df_update<<<df_blocks(n), 256, 0, st>>>(cu, cv, F(q.du), F(q.dv), n);
            launches++;
        }
    }
    dm_count_launches(launches);
    if ((e = cudaMemcpyAsync(out_u, cu, (size_t)W * H * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out_v, cv, (size_t)W * H * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    return cudaGetLastError();
}

