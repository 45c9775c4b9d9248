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
// The SOR sweeps are sequential in time (each half-sweep needs the other
// colour's previous values), so the launch count, not the arithmetic, bounds
// the solver: the smallest levels (up to 1024 pixels) run entirely in one
// CTA with their state in shared memory; larger levels run 8 half-sweeps per launch, temporally blocked in
// shared memory (a tile plus an 8-pixel halo), which gives the same bits as
// 8 global half-sweeps.
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

// The fixed-point step's arithmetic for one pixel, on values: the
// smoothness weight from the forward differences of u + du, v + dv (has_r /
// has_d: the right / lower neighbour exists), the data and matching weights
// and the 2x2 system (A11, A12, A22, b1, b2).
struct DfPix {
    float ps, a11, a12, a22, b1, b2;
};

__device__ __forceinline__ DfPix df_weights_vals(float u, float du, float v, float dv, bool has_r, float ur, float dur,
                                                 float vr, float dvr, bool has_d, float ud, float dud, float vd, float dvd,
                                                 const float* d, float alpha, float mc, float mu, float mv,
                                                 const DfConst& k) {
    const float U = __fadd_rn(u, du), V = __fadd_rn(v, dv);
    float ux = 0.0f, uy = 0.0f, vx = 0.0f, vy = 0.0f;
    if (has_r) {
        ux = __fsub_rn(__fadd_rn(ur, dur), U);
        vx = __fsub_rn(__fadd_rn(vr, dvr), V);
    }
    if (has_d) {
        uy = __fsub_rn(__fadd_rn(ud, dud), U);
        vy = __fsub_rn(__fadd_rn(vd, dvd), V);
    }
    DfPix r;
    const float s2 = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy)), __fmul_rn(vx, vx)), __fmul_rn(vy, vy));
    r.ps = __fmul_rn(alpha, df_dpsi(s2, k.eps2));
    const float d0 = d[0], d1 = d[1], d2 = d[2], d3 = d[3], d4 = d[4], d5 = d[5], d6 = d[6], d7 = d[7], d8 = d[8];
    const float d9 = d[9], d10 = d[10];
    float a0 = 0.0f;
    if (k.delta > 0.0f) {
        const float r0 = __fadd_rn(__fadd_rn(__fmul_rn(d0, du), __fmul_rn(d1, dv)), d2);
        a0 = __fmul_rn(__fmul_rn(k.delta, df_dpsi(__fmul_rn(d8, __fmul_rn(r0, r0)), k.eps2)), d8);
    }
    const float rx = __fadd_rn(__fadd_rn(__fmul_rn(d3, du), __fmul_rn(d4, dv)), d6);
    const float ry = __fadd_rn(__fadd_rn(__fmul_rn(d4, du), __fmul_rn(d5, dv)), d7);
    const float ag = __fmul_rn(k.gamma, df_dpsi(__fadd_rn(__fmul_rn(d9, __fmul_rn(rx, rx)), __fmul_rn(d10, __fmul_rn(ry, ry))), k.eps2));
    float mw = 0.0f;
    if (mc > 0.0f) {
        const float eu = __fsub_rn(U, mu), ev = __fsub_rn(V, mv);
        mw = __fmul_rn(mc, df_dpsi(__fadd_rn(__fmul_rn(eu, eu), __fmul_rn(ev, ev)), k.eps2));
    }
    const float gx = __fmul_rn(ag, d9), gy = __fmul_rn(ag, d10);
    const float a0x = __fmul_rn(a0, d0), a0y = __fmul_rn(a0, d1);
    r.a11 = __fadd_rn(__fadd_rn(__fmul_rn(a0x, d0), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d3), __fmul_rn(__fmul_rn(gy, d4), d4))), mw);
    r.a12 = __fadd_rn(__fmul_rn(a0x, d1), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d4), __fmul_rn(__fmul_rn(gy, d4), d5)));
    r.a22 = __fadd_rn(__fadd_rn(__fmul_rn(a0y, d1), __fadd_rn(__fmul_rn(__fmul_rn(gx, d4), d4), __fmul_rn(__fmul_rn(gy, d5), d5))), mw);
    r.b1 = __fsub_rn(-__fadd_rn(__fmul_rn(a0x, d2), __fadd_rn(__fmul_rn(__fmul_rn(gx, d3), d6), __fmul_rn(__fmul_rn(gy, d4), d7))),
                     __fmul_rn(mw, __fsub_rn(u, mu)));
    r.b2 = __fsub_rn(-__fadd_rn(__fmul_rn(a0y, d2), __fadd_rn(__fmul_rn(__fmul_rn(gx, d4), d6), __fmul_rn(__fmul_rn(gy, d5), d7))),
                     __fmul_rn(mw, __fsub_rn(v, mv)));
    return r;
}

__device__ __forceinline__ void df_load_d(const float* D, long long n, long long o, float* d) {
#pragma unroll
    for (int j = 0; j < 11; j++) d[j] = D[j * n + o];
}

__device__ __forceinline__ void df_weights_at(const DfLevel& L, const DfConst& k, long long o) {
    const int x = (int)(o % L.w), y = (int)(o / L.w);
    const bool hr = x + 1 < L.w, hd = y + 1 < L.h;
    const long long r = hr ? o + 1 : o, dn = hd ? o + L.w : o;
    float d[11];
    df_load_d(L.D, L.n, o, d);
    const DfPix q = df_weights_vals(L.u[o], L.du[o], L.v[o], L.dv[o], hr, L.u[r], L.du[r], L.v[r], L.dv[r], hd, L.u[dn],
                                    L.du[dn], L.v[dn], L.dv[dn], d, L.alpha[o], L.mc[o], L.mu[o], L.mv[o], k);
    const long long n = L.n;
    L.ps[o] = q.ps;
    L.A[o] = q.a11;
    L.A[n + o] = q.a12;
    L.A[2 * n + o] = q.a22;
    L.A[3 * n + o] = q.b1;
    L.A[4 * n + o] = q.b2;
}

// One SOR relaxation of a pixel from its existing 4-neighbours (left, right,
// up, down, compacted into nb[0..nn)): edge weight (ps_o + ps_p) / 2,
//   du = (1 - omega) du + omega (b1 + sum w (du_p + u_p - u_o) - A12 dv) / (A11 + sum w),
// then dv the same way with the new du.  Get(p, ps, du, u, dv, v) reads a neighbour.
template <class Get>
__device__ __forceinline__ void df_sor_vals(int nn, const int* nb, Get get, float pso, float uo, float vo, float a11,
                                            float a12, float a22, float b1, float b2, const DfConst& k, float& du,
                                            float& dv) {
    float sw = 0.0f, su = 0.0f, sv = 0.0f;
    for (int j = 0; j < nn; j++) {
        float psp, dup, up, dvp, vp;
        get(nb[j], psp, dup, up, dvp, vp);
        const float we = __fmul_rn(0.5f, __fadd_rn(pso, psp));
        sw = __fadd_rn(sw, we);
        su = __fadd_rn(su, __fmul_rn(we, __fsub_rn(__fadd_rn(dup, up), uo)));
        sv = __fadd_rn(sv, __fmul_rn(we, __fsub_rn(__fadd_rn(dvp, vp), vo)));
    }
    const float nu = __fsub_rn(__fadd_rn(b1, su), __fmul_rn(a12, dv));
    du = __fadd_rn(__fmul_rn(k.one_m_omega, du), __fmul_rn(k.omega, __fdiv_rn(nu, __fadd_rn(a11, sw))));
    const float nv = __fsub_rn(__fadd_rn(b2, sv), __fmul_rn(a12, du));
    dv = __fadd_rn(__fmul_rn(k.one_m_omega, dv), __fmul_rn(k.omega, __fdiv_rn(nv, __fadd_rn(a22, sw))));
}

__global__ void k_df_weights(DfLevel L, DfConst k) {
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < L.n; o += (long long)gridDim.x * blockDim.x)
        df_weights_at(L, k, o);
}

// Temporally blocked red-black SOR: a CTA owns a TB_W x TB_H tile and stages
// it with a halo of S pixels (S = the half-sweeps of this launch, <= TB_S) in
// shared memory, then runs S half-sweeps there, colour start, start + 1, ...
// Half-sweep j updates the pixels of its colour in the staged region shrunk by
// j + 1 on every side that is not the image border: their neighbours then
// hold exactly the values the global sweep would give them, so after S
// half-sweeps the tile itself is exact and is written back -- the same bits
// as S global half-sweeps, with one launch and no global barrier between them.
// The halos of other CTAs overlap this tile, so the increments are read from
// L.du / L.dv and written to a second pair of buffers (ping-pong between
// launches): no CTA ever sees another's updates of the same launch.
constexpr int TB_W = 32, TB_H = 16, TB_S = 8;
constexpr int TB_LW = TB_W + 2 * TB_S, TB_LH = TB_H + 2 * TB_S, TB_LN = TB_LW * TB_LH;
constexpr size_t TB_SMEM = (size_t)TB_LN * 10 * sizeof(float);

constexpr int TB_THREADS = 1024;                  // a tile's half-sweep is short: many threads, short latency

__global__ void __launch_bounds__(TB_THREADS) k_df_sor_tb(DfLevel L, DfConst k, int start_color, int S, float* __restrict__ out_du,
                                                   float* __restrict__ out_dv) {
    extern __shared__ __align__(16) float sm[];
    float* sdu = sm;
    float* sdv = sm + TB_LN;
    float* su_ = sm + 2 * TB_LN;
    float* sv_ = sm + 3 * TB_LN;
    float* sps = sm + 4 * TB_LN;
    float* sA = sm + 5 * TB_LN;          // [5][TB_LN]
    const int tiles_x = (L.w + TB_W - 1) / TB_W;
    const int tx0 = (blockIdx.x % tiles_x) * TB_W, ty0 = (blockIdx.x / tiles_x) * TB_H;
    const int tx1 = min(tx0 + TB_W, L.w), ty1 = min(ty0 + TB_H, L.h);
    const int lx0 = max(tx0 - S, 0), ly0 = max(ty0 - S, 0);
    const int lx1 = min(tx1 + S, L.w), ly1 = min(ty1 + S, L.h);
    const int lw = lx1 - lx0, lh = ly1 - ly0, ln = lw * lh;
    const long long n = L.n;
    for (int i = threadIdx.x; i < ln; i += blockDim.x) {
        const long long o = (long long)(ly0 + i / lw) * L.w + (lx0 + i % lw);
        sdu[i] = L.du[o];
        sdv[i] = L.dv[o];
        su_[i] = L.u[o];
        sv_[i] = L.v[o];
        sps[i] = L.ps[o];
#pragma unroll
        for (int j = 0; j < 5; j++) sA[j * TB_LN + i] = L.A[j * n + o];
    }
    __syncthreads();
    auto get = [&](int p, float& ps, float& du, float& u, float& dv, float& v) {
        ps = sps[p]; du = sdu[p]; u = su_[p]; dv = sdv[p]; v = sv_[p];
    };
    for (int j = 0; j < S; j++) {
        const int color = (start_color + j) & 1;
        const int ax0 = lx0 > 0 ? lx0 + j + 1 : lx0, ay0 = ly0 > 0 ? ly0 + j + 1 : ly0;
        const int ax1 = lx1 < L.w ? lx1 - j - 1 : lx1, ay1 = ly1 < L.h ? ly1 - j - 1 : ly1;
        const int aw = ax1 - ax0, ah = ay1 - ay0;
        if (aw > 0 && ah > 0) {
            const int half = (aw + 1) / 2;
            for (int i = threadIdx.x; i < half * ah; i += blockDim.x) {
                const int gy = ay0 + i / half;
                const int gx = ax0 + 2 * (i % half) + ((gy + ax0 + color) & 1);
                if (gx >= ax1) continue;
                const int p = (gy - ly0) * lw + (gx - lx0);
                int nb[4], nn = 0;
                if (gx > 0) nb[nn++] = p - 1;
                if (gx + 1 < L.w) nb[nn++] = p + 1;
                if (gy > 0) nb[nn++] = p - lw;
                if (gy + 1 < L.h) nb[nn++] = p + lw;
                float du = sdu[p], dv = sdv[p];
                df_sor_vals(nn, nb, get, sps[p], su_[p], sv_[p], sA[p], sA[TB_LN + p], sA[2 * TB_LN + p],
                            sA[3 * TB_LN + p], sA[4 * TB_LN + p], k, du, dv);
                sdu[p] = du;
                sdv[p] = dv;
            }
        }
        __syncthreads();
    }
    const int ow = tx1 - tx0;
    for (int i = threadIdx.x; i < ow * (ty1 - ty0); i += blockDim.x) {
        const int gx = tx0 + i % ow, gy = ty0 + i / ow;
        const int p = (gy - ly0) * lw + (gx - lx0);
        const long long o = (long long)gy * L.w + gx;
        out_du[o] = sdu[p];
        out_dv[o] = sdv[p];
    }
}

__global__ void k_df_update(float* __restrict__ u, float* __restrict__ v, const float* __restrict__ du,
                            const float* __restrict__ dv, long long n) {
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < n; o += (long long)gridDim.x * blockDim.x) {
        u[o] = __fadd_rn(u[o], du[o]);
        v[o] = __fadd_rn(v[o], dv[o]);
    }
}

// A whole small level in one CTA with its state in shared memory: u, v, du,
// dv, ps and the system (10 floats per pixel); n_fixed x (weights, then
// n_sor red-black sweeps) with block barriers between the passes, then
// w += dw.  The same per-pixel arithmetic as the multi-launch path.
constexpr int DF_SMALL_THREADS = 1024;
// Pixels of a level solved by one CTA: above about a thousand pixels a single
// SM is slower than the blocked launches (1024x436 pair: 43.0 ms with 5120
// and 256-thread blocked CTAs, 39.4 ms with 1024 and 1024 threads).  At most
// 5120 (200 KB of shared memory).
constexpr int DF_SMALL_MAX = 1024;
constexpr size_t DF_SMALL_SMEM = (size_t)DF_SMALL_MAX * 10 * sizeof(float);
static_assert(DF_SMALL_MAX <= 5120, "small-level state must fit shared memory");

__global__ void __launch_bounds__(DF_SMALL_THREADS) k_df_level_small(DfLevel L, DfConst k, int n_fixed, int n_sor) {
    extern __shared__ __align__(16) float sm[];
    const int n = (int)L.n, w = L.w, h = L.h;
    float* su_ = sm;
    float* sv_ = sm + n;
    float* sdu = sm + 2 * n;
    float* sdv = sm + 3 * n;
    float* sps = sm + 4 * n;
    float* sA = sm + 5 * n;              // [5][n]
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
        su_[o] = L.u[o];
        sv_[o] = L.v[o];
        sdu[o] = 0.0f;
        sdv[o] = 0.0f;
    }
    __syncthreads();
    auto get = [&](int p, float& ps, float& du, float& u, float& dv, float& v) {
        ps = sps[p]; du = sdu[p]; u = su_[p]; dv = sdv[p]; v = sv_[p];
    };
    const int half = (w + 1) / 2;
    for (int it = 0; it < n_fixed; it++) {
        for (int o = threadIdx.x; o < n; o += blockDim.x) {
            const int x = o % w, y = o / w;
            const bool hr = x + 1 < w, hd = y + 1 < h;
            const int r = hr ? o + 1 : o, dn = hd ? o + w : o;
            float d[11];
            df_load_d(L.D, L.n, o, d);
            const DfPix q = df_weights_vals(su_[o], sdu[o], sv_[o], sdv[o], hr, su_[r], sdu[r], sv_[r], sdv[r], hd, su_[dn],
                                            sdu[dn], sv_[dn], sdv[dn], d, L.alpha[o], L.mc[o], L.mu[o], L.mv[o], k);
            sps[o] = q.ps;
            sA[o] = q.a11;
            sA[n + o] = q.a12;
            sA[2 * n + o] = q.a22;
            sA[3 * n + o] = q.b1;
            sA[4 * n + o] = q.b2;
        }
        __syncthreads();
        for (int s = 0; s < n_sor; s++)
            for (int color = 0; color < 2; color++) {
                for (int i = threadIdx.x; i < half * h; i += blockDim.x) {
                    const int y = i / half;
                    const int x = 2 * (i % half) + ((y + color) & 1);
                    if (x >= w) continue;
                    const int p = y * w + x;
                    int nb[4], nn = 0;
                    if (x > 0) nb[nn++] = p - 1;
                    if (x + 1 < w) nb[nn++] = p + 1;
                    if (y > 0) nb[nn++] = p - w;
                    if (y + 1 < h) nb[nn++] = p + w;
                    float du = sdu[p], dv = sdv[p];
                    df_sor_vals(nn, nb, get, sps[p], su_[p], sv_[p], sA[p], sA[n + p], sA[2 * n + p], sA[3 * n + p],
                                sA[4 * n + p], k, du, dv);
                    sdu[p] = du;
                    sdv[p] = dv;
                }
                __syncthreads();
            }
    }
    float* u = const_cast<float*>(L.u);
    float* v = const_cast<float*>(L.v);
    for (int o = threadIdx.x; o < n; o += blockDim.x) {
        u[o] = __fadd_rn(su_[o], sdu[o]);
        v[o] = __fadd_rn(sv_[o], sdv[o]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: the plan (level sizes, constants, workspace) and the launches.
// ---------------------------------------------------------------------------
namespace {
constexpr double kPi = 3.14159265358979323846;
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
    size_t* one[] = {&q->tmp, &q->fa_u, &q->fa_v, &q->fb_u, &q->fb_v, &q->du, &q->dv, &q->du2, &q->dv2, &q->alpha, &q->I2w, &q->Im,
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
    static std::atomic<unsigned long long> tb_done{0}, small_done{0};
    if ((e = dm_smem_opt_in(reinterpret_cast<const void*>(k_df_sor_tb), (int)TB_SMEM, tb_done)) != cudaSuccess) return e;
    if ((e = dm_smem_opt_in(reinterpret_cast<const void*>(k_df_level_small), (int)DF_SMALL_SMEM, small_done)) != cudaSuccess)
        return e;
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
            k_df_level_small<<<1, DF_SMALL_THREADS, DF_SMALL_SMEM, st>>>(L, k, q.n_fixed, q.n_sor);
            launches++;
        } else {
            const unsigned tiles = (unsigned)(((w + TB_W - 1) / TB_W) * ((h + TB_H - 1) / TB_H));
            float* alt_u = F(q.du2);
            float* alt_v = F(q.dv2);
            for (int it = 0; it < q.n_fixed; it++) {
                k_df_weights<<<df_blocks(n), 256, 0, st>>>(L, k);
                launches++;
                for (int j = 0; j < 2 * q.n_sor; j += TB_S) {
                    const int S = 2 * q.n_sor - j < TB_S ? 2 * q.n_sor - j : TB_S;
                    k_df_sor_tb<<<tiles, TB_THREADS, TB_SMEM, st>>>(L, k, j & 1, S, alt_u, alt_v);
                    launches++;
                    float* t = L.du; L.du = alt_u; alt_u = t;
                    t = L.dv; L.dv = alt_v; alt_v = t;
                }
            }
            k_df_update<<<df_blocks(n), 256, 0, st>>>(cu, cv, L.du, L.dv, n);
            launches++;
        }
    }
    dm_count_launches(launches);
    if ((e = cudaMemcpyAsync(out_u, cu, (size_t)W * H * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(out_v, cv, (size_t)W * H * 4, cudaMemcpyDeviceToDevice, st)) != cudaSuccess) return e;
    return cudaGetLastError();
}

