/*
 * DeepFlow oracle (Sec. 4.3) -- TEST INFRASTRUCTURE ONLY, included at the end
 * of dm_oracle.c (it uses that file's working precision, smoothing and exp).
 *
 * Variational refinement of a flow field w = (u, v) between I1 and I2 with
 * a data term (normalised gradient constancy weighted by gamma, normalised
 * brightness constancy weighted by delta), a locally weighted smoothness term
 * alpha(x) = exp(-kappa |grad I1|) and a matching term beta_k c phi Psi(|w - w'|^2)
 * pulling the flow towards the DeepMatching matches, all with the robust
 * penalizer Psi(s^2) = sqrt(s^2 + eps^2).  Coarse-to-fine with downsampling
 * factor eta, 5 fixed-point iterations per level (the non-linear weights
 * recomputed from the current increment), 25 SOR iterations each.
 *
 * Readings where the paper is silent (each is one choice, used identically
 * by the GPU path):
 *   - intensities are scaled to [0, 255] (as for the descriptors), then
 *     smoothed by a Gaussian of std sigma (taps as for the descriptors);
 *     kappa applies to the gradient norm of the [0, 1] image (|grad| / 255);
 *   - pyramid: level k+1 is level k resampled bilinearly at x_k = (x + 1/2)/eta
 *     - 1/2 (clamped to the image), sizes floor(eta W_k + 1/2); levels stop
 *     before a side falls below min_size;  the flow is carried to the finer
 *     level by bilinear resampling at (x + 1/2) eta - 1/2, divided by eta;
 *   - derivatives: central differences with replicated border on the mean
 *     Im = (I1 + I2(x + w)) / 2 (I2 sampled bilinearly, clamped); Iz = I2w - I1;
 *     second derivatives Ixx = dx(Ix), Ixy = dy(Ix), Iyy = dy(Iy); gradient
 *     differences Ixz = dx(I2w) - dx(I1), Iyz = dy(I2w) - dy(I1);
 *     normalisations theta0 = 1/(Ix^2 + Iy^2 + zeta^2), thetax = 1/(Ixx^2 +
 *     Ixy^2 + zeta^2), thetay = 1/(Ixy^2 + Iyy^2 + zeta^2);
 *   - smoothness: forward differences (0 at the last column / row) for the
 *     weight psi_s = alpha Psi'(|grad(u+du)|^2 + |grad(v+dv)|^2); the weight
 *     between neighbours is the mean of theirs; 4-neighbourhood, no flux
 *     across the border;
 *   - matches: at full resolution, lambda~ = 10 x the smaller eigenvalue of
 *     the 3x3 sum of the gradient products of I1 at x1, Delta = |I1(x1) -
 *     I2(x2)| + |dx I1(x1) - dx I2(x2)| + |dy I1(x1) - dy I2(x2)| (x2 = x1 + w',
 *     the paper's "x - w'" read with w' pointing from I1 to I2); at level k a
 *     match lands on pixel round((x1 + 1/2) eta^k - 1/2) with w' eta^k, the
 *     higher DeepMatching score (then the lower match index) winning a pixel;
 *     beta_k = beta (k / k_max)^b (beta at a single level);
 *   - SOR: red-black order (x + y even first), relaxation omega; per pixel du
 *     is updated first, then dv with the new du.
 */

typedef struct {
    double sigma, eta, gamma, delta, beta, b, kappa, zeta, eps, sigma_m, omega, image_scale;
    int n_fixed, n_sor, min_size;
} df_params;

static df_params df_unpack(const double* p) {
    df_params q;
    q.sigma = p[0]; q.eta = p[1]; q.gamma = p[2]; q.delta = p[3]; q.beta = p[4]; q.b = p[5];
    q.kappa = p[6]; q.zeta = p[7]; q.eps = p[8]; q.sigma_m = p[9]; q.omega = p[10]; q.image_scale = p[11];
    q.n_fixed = (int)p[12]; q.n_sor = (int)p[13]; q.min_size = (int)p[14];
    return q;
}

/* Pyramid sizes: level 0 = W x H; returns the number of levels (k_max + 1). */
int orc_df_levels(int W, int H, const double* prm, int* ws, int* hs, int cap) {
    df_params q = df_unpack(prm);
    int n = 0;
    ws[0] = W; hs[0] = H; n = 1;
    while (n < cap) {
        int w = (int)floor(q.eta * ws[n - 1] + 0.5), h = (int)floor(q.eta * hs[n - 1] + 0.5);
        if (w < q.min_size || h < q.min_size) break;
        ws[n] = w; hs[n] = h; n++;
    }
    return n;
}

/* Bilinear sample of f (W x H) at (xs, ys), coordinates clamped to the image. */
static real df_bilinear(const real* f, int W, int H, real xs, real ys) {
    if (xs < (real)0) xs = (real)0;
    if (ys < (real)0) ys = (real)0;
    if (xs > (real)(W - 1)) xs = (real)(W - 1);
    if (ys > (real)(H - 1)) ys = (real)(H - 1);
    real fx0 = floor(xs), fy0 = floor(ys);
    int x0 = (int)fx0, y0 = (int)fy0;
    int x1 = x0 + 1 < W ? x0 + 1 : W - 1, y1 = y0 + 1 < H ? y0 + 1 : H - 1;
    real fx = xs - fx0, fy = ys - fy0;
    real p00 = f[(size_t)y0 * W + x0], p10 = f[(size_t)y0 * W + x1];
    real p01 = f[(size_t)y1 * W + x0], p11 = f[(size_t)y1 * W + x1];
    real top = p00 + fx * (p10 - p00);
    real bot = p01 + fx * (p11 - p01);
    return top + fy * (bot - top);
}

/* dst (Wd x Hd) = src (Ws x Hs) sampled at (x + 1/2) * s - 1/2 (s = 1/eta
 * going down, eta going up), times `mul`. */
static void df_resample(const real* src, int Ws, int Hs, real* dst, int Wd, int Hd, real s, int down, real mul) {
    for (int y = 0; y < Hd; y++)
        for (int x = 0; x < Wd; x++) {
            real xs = down ? ((real)x + (real)0.5) / s - (real)0.5 : ((real)x + (real)0.5) * s - (real)0.5;
            real ys = down ? ((real)y + (real)0.5) / s - (real)0.5 : ((real)y + (real)0.5) * s - (real)0.5;
            dst[(size_t)y * Wd + x] = df_bilinear(src, Ws, Hs, xs, ys) * mul;
        }
}

static real df_dx(const real* f, int W, int x, int y) {
    return (real)0.5 * (f[(size_t)y * W + (x + 1 < W ? x + 1 : W - 1)] - f[(size_t)y * W + (x > 0 ? x - 1 : 0)]);
}
static real df_dy(const real* f, int W, int H, int x, int y) {
    return (real)0.5 * (f[(size_t)(y + 1 < H ? y + 1 : H - 1) * W + x] - f[(size_t)(y > 0 ? y - 1 : 0) * W + x]);
}

/* Psi'(s2) = 1 / (2 sqrt(s2 + eps^2)). */
static real df_dpsi(real s2, real eps2) { return (real)0.5 / RSQRT(s2 + eps2); }

/* Per-match weight phi at full resolution (presmoothed images in [0,255]). */
static real df_phi(const real* I1, const real* I2, int W1, int H1, int W2, int H2, int x1, int y1, int x2, int y2,
                   real sigma_m) {
    real a = 0, b = 0, c = 0;
    for (int dy = -1; dy <= 1; dy++)
        for (int dx = -1; dx <= 1; dx++) {
            int xx = clampi(x1 + dx, 0, W1 - 1), yy = clampi(y1 + dy, 0, H1 - 1);
            real gx = df_dx(I1, W1, xx, yy), gy = df_dy(I1, W1, H1, xx, yy);
            a = a + gx * gx;
            b = b + gx * gy;
            c = c + gy * gy;
        }
    real h = (a - c) * (real)0.5;
    real lmin = (a + c) * (real)0.5 - RSQRT(h * h + b * b);
    if (lmin < (real)0) lmin = (real)0;
    real lt = (real)10 * lmin;
    real d = (real)fabs((double)(I1[(size_t)y1 * W1 + x1] - I2[(size_t)y2 * W2 + x2]));
    d = d + (real)fabs((double)(df_dx(I1, W1, x1, y1) - df_dx(I2, W2, x2, y2)));
    d = d + (real)fabs((double)(df_dy(I1, W1, H1, x1, y1) - df_dy(I2, W2, H2, x2, y2)));
    const real norm = (real)(1.0 / (sqrt(2.0 * 3.14159265358979323846)));
    real z = -(d / ((real)2 * sigma_m));
    return RSQRT(lt) / sigma_m * norm * REXP(z);
}

/* n_sor red-black SOR sweeps (x + y even first) on the linear system of one
 * fixed-point step: per pixel o, with the coefficients a = A[o][0..4] =
 * (A11, A12, A22, b1, b2) and the edge weight (ps[o] + ps[p]) / 2 to each
 * 4-neighbour p (left, right, up, down),
 *   (A11 + sum_p w_op) du_o + A12 dv_o = b1 + sum_p w_op (du_p + u_p - u_o),
 *   A12 du_o + (A22 + sum_p w_op) dv_o = b2 + sum_p w_op (dv_p + v_p - v_o);
 * du is relaxed first, then dv with the new du. */
static void df_sor(const real* A, const real* ps, const real* u, const real* v, real* du, real* dv, int w, int h,
                   real omega, int n_sor) {
    for (int s = 0; s < n_sor; s++)
        for (int color = 0; color < 2; color++)
            for (int y = 0; y < h; y++)
                for (int x = (y + color) & 1; x < w; x += 2) {
                    size_t o = (size_t)y * w + x;
                    const real* a = A + o * 5;
                    real sw = (real)0, su = (real)0, sv = (real)0;
                    size_t nb[4];
                    int nn = 0;
                    if (x > 0) nb[nn++] = o - 1;
                    if (x + 1 < w) nb[nn++] = o + 1;
                    if (y > 0) nb[nn++] = o - w;
                    if (y + 1 < h) nb[nn++] = o + w;
                    for (int j = 0; j < nn; j++) {
                        size_t p = nb[j];
                        real we = (real)0.5 * (ps[o] + ps[p]);
                        sw = sw + we;
                        su = su + we * ((du[p] + u[p]) - u[o]);
                        sv = sv + we * ((dv[p] + v[p]) - v[o]);
                    }
                    real nu_ = (a[3] + su) - a[1] * dv[o];
                    du[o] = ((real)1 - omega) * du[o] + omega * (nu_ / (a[0] + sw));
                    real nv_ = (a[4] + sv) - a[1] * du[o];
                    dv[o] = ((real)1 - omega) * dv[o] + omega * (nv_ / (a[2] + sw));
                }
}

int orc_df_sor(const real* A, const real* ps, const real* u, const real* v, real* du, real* dv, int w, int h,
               double omega, int n_sor) {
    if (w < 1 || h < 1) return -1;
    df_sor(A, ps, u, v, du, dv, w, h, (real)omega, n_sor);
    return 0;
}

int orc_df_resample(const real* src, int Ws, int Hs, real* dst, int Wd, int Hd, double s, int down, double mul) {
    df_resample(src, Ws, Hs, dst, Wd, Hd, (real)s, down, (real)mul);
    return 0;
}

/* phi of the match (x1, y1) -> (x2, y2) on presmoothed images in [0,255]. */
double orc_df_phi(const real* I1, const real* I2, int W1, int H1, int W2, int H2, int x1, int y1, int x2, int y2,
                  double sigma_m) {
    return (double)df_phi(I1, I2, W1, H1, W2, H2, x1, y1, x2, y2, (real)sigma_m);
}

/* DeepFlow on images I1, I2 (W x H, values in [0,1]) with matches m[n][5]
 * (x1, y1, x2, y2, score), parameters prm (see df_unpack).  u, v: output
 * [H][W].  Returns 0, or -1 on invalid input. */
int orc_deepflow(const float* img1, const float* img2, int W, int H, const float* m, int n, const double* prm,
                 real* u_out, real* v_out) {
    if (W < 1 || H < 1 || n < 0) return -1;
    df_params q = df_unpack(prm);
    int ws[256], hs[256];
    const int nl = orc_df_levels(W, H, prm, ws, hs, 256);
    const int kmax = nl - 1;
    const real eta = (real)q.eta, scale = (real)q.image_scale;
    const real zeta2 = (real)(q.zeta * q.zeta), eps2 = (real)(q.eps * q.eps), omega = (real)q.omega;
    const real gamma = (real)q.gamma, delta = (real)q.delta, kappa = (real)q.kappa;
    real* P1[256];
    real* P2[256];
    /* level 0: scaled and presmoothed */
    real taps[65], tmpw;
    int R = gauss_taps(q.sigma, taps, 65);
    (void)tmpw;
    size_t N0 = (size_t)W * H;
    real* tmp = (real*)malloc(N0 * sizeof(real));
    P1[0] = (real*)malloc(N0 * sizeof(real));
    P2[0] = (real*)malloc(N0 * sizeof(real));
    for (size_t i = 0; i < N0; i++) { P1[0][i] = (real)img1[i] * scale; P2[0][i] = (real)img2[i] * scale; }
    smooth(P1[0], W, H, 1, 0, 1, taps, R, tmp);
    smooth(P2[0], W, H, 1, 0, 1, taps, R, tmp);
    for (int k = 1; k < nl; k++) {
        size_t Nk = (size_t)ws[k] * hs[k];
        P1[k] = (real*)malloc(Nk * sizeof(real));
        P2[k] = (real*)malloc(Nk * sizeof(real));
        df_resample(P1[k - 1], ws[k - 1], hs[k - 1], P1[k], ws[k], hs[k], eta, 1, (real)1);
        df_resample(P2[k - 1], ws[k - 1], hs[k - 1], P2[k], ws[k], hs[k], eta, 1, (real)1);
    }
    /* per-match weights at full resolution */
    real* phi = (real*)malloc((size_t)(n > 0 ? n : 1) * sizeof(real));
    for (int i = 0; i < n; i++) {
        int x1 = clampi((int)m[5 * i], 0, W - 1), y1 = clampi((int)m[5 * i + 1], 0, H - 1);
        int x2 = clampi((int)m[5 * i + 2], 0, W - 1), y2 = clampi((int)m[5 * i + 3], 0, H - 1);
        phi[i] = df_phi(P1[0], P2[0], W, H, W, H, x1, y1, x2, y2, (real)q.sigma_m);
    }
    real* u = NULL;
    real* v = NULL;
    for (int k = kmax; k >= 0; k--) {
        const int w = ws[k], h = hs[k];
        const size_t N = (size_t)w * h;
        real* nu = (real*)calloc(N, sizeof(real));
        real* nv = (real*)calloc(N, sizeof(real));
        if (u) {
            df_resample(u, ws[k + 1], hs[k + 1], nu, w, h, eta, 0, (real)1 / eta);
            df_resample(v, ws[k + 1], hs[k + 1], nv, w, h, eta, 0, (real)1 / eta);
            free(u);
            free(v);
        }
        u = nu;
        v = nv;
        const real* I1 = P1[k];
        const real* I2 = P2[k];
        /* matches on this level */
        const double sk = pow(q.eta, (double)k);
        real* mc = (real*)calloc(N, sizeof(real));     /* beta_k phi at matched pixels, 0 elsewhere */
        real* mu = (real*)calloc(N, sizeof(real));
        real* mv = (real*)calloc(N, sizeof(real));
        int* owner = (int*)malloc(N * sizeof(int));
        for (size_t i = 0; i < N; i++) owner[i] = -1;
        const real beta_k = (real)(kmax > 0 ? q.beta * pow((double)k / (double)kmax, q.b) : q.beta);
        const real skr = (real)sk;
        for (int i = 0; i < n; i++) {
            real fx = ((real)m[5 * i] + (real)0.5) * skr - (real)0.5;
            real fy = ((real)m[5 * i + 1] + (real)0.5) * skr - (real)0.5;
            int px = clampi((int)floor(fx + (real)0.5), 0, w - 1), py = clampi((int)floor(fy + (real)0.5), 0, h - 1);
            size_t o = (size_t)py * w + px;
            int cur = owner[o];
            if (cur < 0 || m[5 * i + 4] > m[5 * cur + 4]) owner[o] = i;
        }
        for (size_t o = 0; o < N; o++) {
            int i = owner[o];
            if (i < 0) continue;
            mc[o] = beta_k * phi[i];
            mu[o] = ((real)m[5 * i + 2] - (real)m[5 * i]) * skr;
            mv[o] = ((real)m[5 * i + 3] - (real)m[5 * i + 1]) * skr;
        }
        free(owner);
        /* alpha and the linearised data term around the current flow */
        real* alpha = (real*)malloc(N * sizeof(real));
        real* Im = (real*)malloc(N * sizeof(real));
        real* I2w = (real*)malloc(N * sizeof(real));
        real* D = (real*)malloc(N * 11 * sizeof(real));   /* Ix Iy Iz Ixx Ixy Iyy Ixz Iyz th0 thx thy */
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t o = (size_t)y * w + x;
                real gx = df_dx(I1, w, x, y) / scale, gy = df_dy(I1, w, h, x, y) / scale;
                alpha[o] = REXP(-(kappa * RSQRT(gx * gx + gy * gy)));
                I2w[o] = df_bilinear(I2, w, h, (real)x + u[o], (real)y + v[o]);
                Im[o] = (real)0.5 * (I1[o] + I2w[o]);
            }
        real* Ixa = (real*)malloc(N * sizeof(real));
        real* Iya = (real*)malloc(N * sizeof(real));
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t o = (size_t)y * w + x;
                Ixa[o] = df_dx(Im, w, x, y);
                Iya[o] = df_dy(Im, w, h, x, y);
            }
        for (int y = 0; y < h; y++)
            for (int x = 0; x < w; x++) {
                size_t o = (size_t)y * w + x;
                real* d = D + o * 11;
                real Ix = Ixa[o], Iy = Iya[o];
                real Ixx = df_dx(Ixa, w, x, y), Ixy = df_dy(Ixa, w, h, x, y), Iyy = df_dy(Iya, w, h, x, y);
                d[0] = Ix; d[1] = Iy; d[2] = I2w[o] - I1[o];
                d[3] = Ixx; d[4] = Ixy; d[5] = Iyy;
                d[6] = df_dx(I2w, w, x, y) - df_dx(I1, w, x, y);
                d[7] = df_dy(I2w, w, h, x, y) - df_dy(I1, w, h, x, y);
                d[8] = (real)1 / ((Ix * Ix + Iy * Iy) + zeta2);
                d[9] = (real)1 / ((Ixx * Ixx + Ixy * Ixy) + zeta2);
                d[10] = (real)1 / ((Ixy * Ixy + Iyy * Iyy) + zeta2);
            }
        free(Ixa); free(Iya); free(Im); free(I2w);
        real* du = (real*)calloc(N, sizeof(real));
        real* dv = (real*)calloc(N, sizeof(real));
        real* A = (real*)malloc(N * 5 * sizeof(real));    /* A11 A12 A22 b1 b2 */
        real* ps = (real*)malloc(N * sizeof(real));       /* smoothness weight psi_s per pixel */
        for (int it = 0; it < q.n_fixed; it++) {
            for (int y = 0; y < h; y++)
                for (int x = 0; x < w; x++) {
                    size_t o = (size_t)y * w + x;
                    const real* d = D + o * 11;
                    /* smoothness weight: forward differences of u + du, v + dv */
                    real U = u[o] + du[o], V = v[o] + dv[o];
                    real ux = (real)0, uy = (real)0, vx = (real)0, vy = (real)0;
                    if (x + 1 < w) { ux = (u[o + 1] + du[o + 1]) - U; vx = (v[o + 1] + dv[o + 1]) - V; }
                    if (y + 1 < h) { uy = (u[o + w] + du[o + w]) - U; vy = (v[o + w] + dv[o + w]) - V; }
                    ps[o] = alpha[o] * df_dpsi(((ux * ux + uy * uy) + vx * vx) + vy * vy, eps2);
                    /* data term weights */
                    real r0 = (d[0] * du[o] + d[1] * dv[o]) + d[2];
                    real a0 = delta > (real)0 ? (delta * df_dpsi(d[8] * (r0 * r0), eps2)) * d[8] : (real)0;
                    real rx = (d[3] * du[o] + d[4] * dv[o]) + d[6];
                    real ry = (d[4] * du[o] + d[5] * dv[o]) + d[7];
                    real ag = gamma * df_dpsi(d[9] * (rx * rx) + d[10] * (ry * ry), eps2);
                    real mw = (real)0;
                    if (mc[o] > (real)0) {
                        real eu = U - mu[o], ev = V - mv[o];
                        mw = mc[o] * df_dpsi(eu * eu + ev * ev, eps2);
                    }
                    real* a = A + o * 5;
                    real gx_ = ag * d[9], gy_ = ag * d[10];
                    a[0] = ((a0 * d[0]) * d[0] + ((gx_ * d[3]) * d[3] + (gy_ * d[4]) * d[4])) + mw;
                    a[1] = (a0 * d[0]) * d[1] + ((gx_ * d[3]) * d[4] + (gy_ * d[4]) * d[5]);
                    a[2] = ((a0 * d[1]) * d[1] + ((gx_ * d[4]) * d[4] + (gy_ * d[5]) * d[5])) + mw;
                    a[3] = -((a0 * d[0]) * d[2] + ((gx_ * d[3]) * d[6] + (gy_ * d[4]) * d[7])) - mw * (u[o] - mu[o]);
                    a[4] = -((a0 * d[1]) * d[2] + ((gx_ * d[4]) * d[6] + (gy_ * d[5]) * d[7])) - mw * (v[o] - mv[o]);
                }
            df_sor(A, ps, u, v, du, dv, w, h, omega, q.n_sor);
        }
        for (size_t o = 0; o < N; o++) { u[o] = u[o] + du[o]; v[o] = v[o] + dv[o]; }
        free(du); free(dv); free(A); free(ps); free(D); free(alpha); free(mc); free(mu); free(mv);
    }
    memcpy(u_out, u, N0 * sizeof(real));
    memcpy(v_out, v, N0 * sizeof(real));
    free(u); free(v); free(phi); free(tmp);
    for (int k = 0; k < nl; k++) { free(P1[k]); free(P2[k]); }
    return 0;
}
