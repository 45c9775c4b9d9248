/*
 * DeepMatching CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised CPU implementation of the hot path
 * of DeepMatching (Revaud et al., "DeepMatching: Hierarchical Deformable Dense
 * Matching"), written from the paper: pixel descriptors (Sec. 3.2), bottom
 * level correlation (Eq. 3-4), the bottom-up pyramid (Eq. 5-12 and
 * Algorithm 1, boundary rule of Sec. 3.2), top-down backtracking with merging
 * (Eq. 13-15) and reciprocal verification (Eq. 16); the DM* backtracking
 * variant's level maps (Sec. 5.3); and DeepFlow (Sec. 4.3, df_oracle.c).
 *
 * Only the test-suite, the smoke check and the CPU-baseline leg of the bench
 * may load this file's library.  It shares no source with the CUDA path.
 *
 * The file is compiled twice:
 *   ORC_F32 = 0 : FP64, the method in the paper's own order (Algorithm 1
 *                 rectifies every map value, then max-pools).
 *   ORC_F32 = 1 : FP32 "canonical mirror": the same method with one fixed
 *                 operation order (stated at each step), own exp/log/pow
 *                 routines, max-pooling on the raw aggregate followed by the
 *                 power (equal to the paper's order because x -> x^lambda is
 *                 increasing on [0,1]), 4-child sums in child order
 *                 (compensated with Knuth's TwoSum by default, plain on
 *                 request), and path scores accumulated exactly in unsigned
 *                 32-bit fixed point with 28 fractional bits (each term
 *                 rounded to the nearest multiple of 2^-28, the sum rounded
 *                 to FP32 once at the end).  It is the bit-exact target of
 *                 the FP32 GPU path.
 *
 * Readings of the paper where it is silent or ambiguous:
 *   - Gaussian "radius" nu = standard deviation; taps on [-ceil(3nu), ceil(3nu)],
 *       renormalised to sum 1; replicate border; nu = 0 is the identity.
 *   - gradient = central differences, replicate border.
 *   - images come in [0,1] and are multiplied by image_scale (255).
 *   - 8 orientations k*pi/4, k = 0..7; channel = max(0, <g, dir_k>).
 *   - mu is appended first, then the 9-vector is L2-normalised.
 *   - image-2 window at pixel t covers [t-2, t+1]^2; zero descriptor outside.
 *   - atomic centres 4k+2 <= W-1.
 *   - a level-N patch exists if at least one child exists; average over valid
 *       children (weight 1/n_valid).
 *   - Theta_i has radius N/8 (a 3x3 max on the child's subsampled grid).
 *   - child i is sampled at q + o_i (sign of Eq. 6 and Eq. 13).
 *   - map domain at level l is ceil(W'/2^l) x ceil(H'/2^l); pooling only over
 *       in-domain positions; a child sample outside the domain contributes 0.
 *   - argmax = first strict maximum, scan order m_y = -1..1 then m_x = -1..1;
 *       ties in BestAt/BestAt': higher score, then lower index.
 *   - L = min{l : 4*2^l >= max(W,H)} (image 1), the level at which Algorithm 1's
 *       loop stops; when image 1 has no patch at that level (a wide, low image:
 *       every child of level l lies 2^l px away, above and below), the top is
 *       the highest level that has a patch, the top of the pyramid the loop
 *       returns; entries = all top positions.
 *   - path score = top value + pooled values along the path, summed top-down
 *       (FP32 mirror: exact fixed-point sum, see the path-score helpers).
 *   - BestAt / BestAt' over aligned 4x4 cells (the atomic patch in I, the cell
 *       floor(t/4) in I'); a tuple survives iff it is the best of both.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORC_F32
#error "compile with -DORC_F32=0 (FP64) or -DORC_F32=1 (FP32 canonical mirror)"
#endif

#if ORC_F32
typedef float real;
#define RFMA(a, b, c) fmaf((a), (b), (c))
#define RSQRT(x) sqrtf(x)
#define RNEG_INF (-INFINITY)
#else
typedef double real;
#define RFMA(a, b, c) fma((a), (b), (c))
#define RSQRT(x) sqrt(x)
#define RNEG_INF (-INFINITY)
#endif

#define ORC_MAXL 30

int orc_real_size(void) { return (int)sizeof(real); }

/* ------------------------------------------------------------------------- */
/* Geometry (Sec. 3.2: G_4, Eq. 7 lattices, Algorithm 1 loop bound)          */
/* ------------------------------------------------------------------------- */

typedef struct {
    int W1, H1, W2, H2;
    int L;            /* number of aggregation iterations */
    int P0x, P0y;     /* atomic grid G_4: centres 4k+2 */
    int Lx, Ly;       /* lattice 4Z^2 inside image 1, patches of levels >= 1 */
    int dw[ORC_MAXL + 2], dh[ORC_MAXL + 2]; /* map domain of level l */
} geom;

static int ceil_half(int v) { return (v + 1) / 2; }

/* Along one axis: does some lattice column (row) hold a patch of level l?
 * n0 atomic columns (all exist), n lattice columns; the children of lattice
 * column i are atomic columns i-1, i at level 1 and lattice columns i -+
 * 2^(l-2) at level l >= 2. */
static int axis_has_patch(int n0, int n, int l) {
    uint8_t* a = (uint8_t*)malloc((size_t)n);
    uint8_t* b = (uint8_t*)malloc((size_t)n);
    int any = 0;
    if (a && b) {
        for (int i = 0; i < n; i++) a[i] = (uint8_t)((i - 1 >= 0 && i - 1 < n0) || i < n0);
        for (int k = 2; k <= l; k++) {
            int s = 1 << (k - 2);
            for (int i = 0; i < n; i++) b[i] = (uint8_t)((i - s >= 0 && a[i - s]) || (i + s < n && a[i + s]));
            memcpy(a, b, (size_t)n);
        }
        for (int i = 0; i < n; i++) any |= a[i];
    }
    free(a);
    free(b);
    return any;
}

static int make_geom(int W1, int H1, int W2, int H2, geom* g) {
    memset(g, 0, sizeof(*g));
    if (W1 < 4 || H1 < 4 || W2 < 1 || H2 < 1) return -1;
    g->W1 = W1; g->H1 = H1; g->W2 = W2; g->H2 = H2;
    int mx = W1 > H1 ? W1 : H1;
    int L = 0;
    long N = 4;
    while (N < mx) { N *= 2; L++; }
    if (L < 1 || L > ORC_MAXL) return -1;
    g->P0x = (W1 - 3) / 4 + 1;
    g->P0y = (H1 - 3) / 4 + 1;
    g->Lx = (W1 - 1) / 4 + 1;
    g->Ly = (H1 - 1) / 4 + 1;
    /* the highest level <= L with a patch: a patch exists iff one of its
     * children does (Eq. 7, boundary rule), and since the four children are
     * the combinations of two columns and two rows, existence is a column
     * condition times a row condition -- check each axis on its own */
    int top = L;
    while (top > 1 && !(axis_has_patch(g->P0x, g->Lx, top) && axis_has_patch(g->P0y, g->Ly, top))) top--;
    g->L = top;
    g->dw[0] = W2; g->dh[0] = H2;
    for (int l = 1; l <= L + 1; l++) { g->dw[l] = ceil_half(g->dw[l - 1]); g->dh[l] = ceil_half(g->dh[l - 1]); }
    return 0;
}

/* out = [L, P0x, P0y, Lx, Ly, dw[0..L+1], dh[0..L+1]] ; returns 0 or -1 */
int orc_geometry(int W1, int H1, int W2, int H2, int* out) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    out[0] = g.L; out[1] = g.P0x; out[2] = g.P0y; out[3] = g.Lx; out[4] = g.Ly;
    for (int l = 0; l <= g.L + 1; l++) { out[5 + l] = g.dw[l]; out[5 + (g.L + 2) + l] = g.dh[l]; }
    return 0;
}

static int npatch(const geom* g, int l) { return l == 0 ? g->P0x * g->P0y : g->Lx * g->Ly; }

/* Child i of patch (ix, iy) at level l >= 1 (Eq. 5: offset (N/4) o_i = 2^l o_i).
 * o_0 = (-1,-1), o_1 = (-1,+1), o_2 = (+1,-1), o_3 = (+1,+1), as (x, y).
 * Returns the child's index at level l-1, or -1 if it lies outside the grid. */
static int child_index(const geom* g, int l, int ix, int iy, int i) {
    int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
    int cx, cy;
    if (l == 1) {                          /* centre 4ix + 2ox -> atomic index (c - 2)/4 */
        cx = ix + (ox - 1) / 2; cy = iy + (oy - 1) / 2;
        if (cx < 0 || cy < 0 || cx >= g->P0x || cy >= g->P0y) return -1;
        return cy * g->P0x + cx;
    }
    int s = 1 << (l - 2);                 /* centre 4ix + 2^l ox -> lattice index ix + 2^(l-2) ox */
    cx = ix + ox * s; cy = iy + oy * s;
    if (cx < 0 || cy < 0 || cx >= g->Lx || cy >= g->Ly) return -1;
    return cy * g->Lx + cx;
}

/* ------------------------------------------------------------------------- */
/* Elementary functions.                                                      */
/* FP64: the C library.  FP32 mirror: own routines with a fixed sequence of   */
/* correctly rounded float operations, so that an independent implementation  */
/* following the same recipe reproduces them bit for bit.                     */
/* ------------------------------------------------------------------------- */
#if ORC_F32
static float f_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t bits_from_f(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* 2^n for n in [-126, 127] built from the exponent field. */
static float pow2i(int n) { return f_from_bits((uint32_t)(n + 127) << 23); }

/* e^z for z <= 0 (clamped at -87).  Cody-Waite reduction z = n ln2 + r with
 * ln2 split into a 16-bit head (exact products n*head) and a tail, then the
 * degree-7 Taylor polynomial of e^r, |r| <= ln2/2, in Horner form. */
static float orc_expf(float z) {
    if (z < -87.0f) z = -87.0f;
    float n = rintf(z * 1.44269504f);
    float r = fmaf(n, -0.693145751953125f, z);
    r = fmaf(n, -1.42860682e-06f, r);
    float p = 1.98412698e-04f;              /* 1/7! */
    p = fmaf(p, r, 1.38888889e-03f);        /* 1/6! */
    p = fmaf(p, r, 8.33333333e-03f);        /* 1/5! */
    p = fmaf(p, r, 4.16666667e-02f);        /* 1/4! */
    p = fmaf(p, r, 1.66666667e-01f);        /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    return p * pow2i((int)n);
}

/* x^lam for x in [0, 1], lam > 0.  x = m 2^e with m in [sqrt(1/2), sqrt(2)];
 * log2 m = (2/ln2) atanh(f), f = (m-1)/(m+1), odd series to f^13;
 * lam*e is split exactly (head + fma residual); 2^g, |g| <= 1/2, by the
 * degree-7 Taylor polynomial of e^(g ln2). */
static float orc_powf(float x, float lam) {
    if (!(x > 0.0f)) return 0.0f;
    int eadj = 0;
    if (x < 1.17549435e-38f) { x = x * 16777216.0f; eadj = -24; }   /* subnormal input */
    uint32_t b = bits_from_f(x);
    int e = (int)((b >> 23) & 0xffu) - 127 + eadj;
    float m = f_from_bits((b & 0x7fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e = e + 1; }
    float f = (m - 1.0f) / (m + 1.0f);
    float f2 = f * f;
    float s = 7.69230769e-02f;               /* 1/13 */
    s = fmaf(s, f2, 9.09090909e-02f);       /* 1/11 */
    s = fmaf(s, f2, 1.11111111e-01f);       /* 1/9 */
    s = fmaf(s, f2, 1.42857143e-01f);       /* 1/7 */
    s = fmaf(s, f2, 2.00000000e-01f);       /* 1/5 */
    s = fmaf(s, f2, 3.33333333e-01f);       /* 1/3 */
    s = fmaf(s, f2, 1.0f);
    float l2m = (2.88539008f * f) * s;      /* 2/ln2 * f * s */
    float fe = (float)e;
    float a = lam * fe;
    float aerr = fmaf(lam, fe, -a);
    float n1 = rintf(a);
    float g = ((a - n1) + aerr) + lam * l2m;
    float n2 = rintf(g);
    g = g - n2;
    float p = 1.52527338e-05f;               /* ln2^7/7! */
    p = fmaf(p, g, 1.54035304e-04f);        /* ln2^6/6! */
    p = fmaf(p, g, 1.33335581e-03f);        /* ln2^5/5! */
    p = fmaf(p, g, 9.61812911e-03f);        /* ln2^4/4! */
    p = fmaf(p, g, 5.55041087e-02f);        /* ln2^3/3! */
    p = fmaf(p, g, 2.40226507e-01f);        /* ln2^2/2! */
    p = fmaf(p, g, 6.93147181e-01f);        /* ln2 */
    p = fmaf(p, g, 1.0f);
    int nt = (int)n1 + (int)n2;
    if (nt < -149 - 2) return 0.0f;
    int na = nt / 2, nb = nt - na;
    return (p * pow2i(na)) * pow2i(nb);
}
#define REXP(z) orc_expf(z)
#define RPOW(x, l) orc_powf((x), (l))
#else
#define REXP(z) exp(z)
#define RPOW(x, l) pow((x), (l))
#endif

/* exported for the accuracy pin of the FP32 routines */
double orc_pow_r(double x, double lam) { return (double)RPOW((real)x, (real)lam); }
/* out[i] = x[i]^lam in the working precision (the rectification of Eq. 11). */
void orc_pow_vec(const real* x, long long n, double lam, real* out) {
    for (long long i = 0; i < n; i++) out[i] = RPOW(x[i], (real)lam);
}
double orc_exp_r(double z) { return (double)REXP((real)z); }

/* ------------------------------------------------------------------------- */
/* Pixel descriptors (Sec. 3.2 "Pixel descriptor"; parameters of Sec. 5.2)    */
/* ------------------------------------------------------------------------- */

/* Gaussian taps of standard deviation nu, computed in double and
 * rounded once to the working precision.  Returns the radius R (0 = identity). */
static int gauss_taps(double nu, real* w, int cap) {
    if (!(nu > 0.0)) { w[0] = (real)1.0; return 0; }
    int R = (int)ceil(3.0 * nu);
    if (2 * R + 1 > cap) R = (cap - 1) / 2;
    double t[65], sum = 0.0;
    for (int j = -R; j <= R; j++) { t[j + R] = exp(-(double)(j * j) / (2.0 * nu * nu)); sum += t[j + R]; }
    for (int j = 0; j <= 2 * R; j++) w[j] = (real)(t[j] / sum);
    return R;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Separable smoothing of nch interleaved channels: horizontal pass, then
 * vertical; each output is acc = fma(w_j, in_j, acc) for j = -R..R from 0. */
static void smooth(real* buf, int W, int H, int nch, int ch0, int chn, const real* w, int R, real* tmp) {
    if (R == 0) return;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = ch0; c < ch0 + chn; c++) {
                real acc = 0;
                for (int j = -R; j <= R; j++)
                    acc = RFMA(w[j + R], buf[((size_t)y * W + clampi(x + j, 0, W - 1)) * nch + c], acc);
                tmp[((size_t)y * W + x) * nch + c] = acc;
            }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            for (int c = ch0; c < ch0 + chn; c++) {
                real acc = 0;
                for (int j = -R; j <= R; j++)
                    acc = RFMA(w[j + R], tmp[((size_t)clampi(y + j, 0, H - 1) * W + x) * nch + c], acc);
                buf[((size_t)y * W + x) * nch + c] = acc;
            }
}

/* cfg = {nu1, nu2, nu3, slope, mu, image_scale}.  out: [H][W][9]. */
int orc_descriptors(const float* img, int W, int H, const double* cfg, real* out) {
    if (W < 1 || H < 1) return -1;
    const real slope = (real)cfg[3], mu = (real)cfg[4], scale = (real)cfg[5];
    real w1[65], w2[65], w3[65];
    int R1 = gauss_taps(cfg[0], w1, 65), R2 = gauss_taps(cfg[1], w2, 65), R3 = gauss_taps(cfg[2], w3, 65);
    size_t n = (size_t)W * H;
    real* s = (real*)malloc(n * sizeof(real));
    real* o = (real*)malloc(n * 8 * sizeof(real));
    real* tmp = (real*)malloc(n * 8 * sizeof(real));
    if (!s || !o || !tmp) { free(s); free(o); free(tmp); return -2; }
    for (size_t i = 0; i < n; i++) s[i] = (real)img[i] * scale;          /* c3 */
    smooth(s, W, H, 1, 0, 1, w1, R1, tmp);                                 /* nu1 */
    /* 8 orientations: exact direction table, r = sqrt(1/2) */
    const real r = (real)0.70710678118654752;
    const real dc[8] = {1, r, 0, -r, -1, -r, 0, r};
    const real ds[8] = {0, r, 1, r, 0, -r, -1, -r};
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            real gx = (s[(size_t)y * W + clampi(x + 1, 0, W - 1)] - s[(size_t)y * W + clampi(x - 1, 0, W - 1)]) * (real)0.5;
            real gy = (s[(size_t)clampi(y + 1, 0, H - 1) * W + x] - s[(size_t)clampi(y - 1, 0, H - 1) * W + x]) * (real)0.5;
            for (int k = 0; k < 8; k++) {
                real v = RFMA(gx, dc[k], gy * ds[k]);
                o[((size_t)y * W + x) * 8 + k] = v > 0 ? v : (real)0;
            }
        }
    smooth(o, W, H, 8, 0, 8, w2, R2, tmp);                                 /* nu2 */
    for (size_t i = 0; i < n * 8; i++) {                                   /* sigmoid cap */
        real t = slope * o[i];
        real e = REXP(-t);
        real d = (real)1 + e;
        o[i] = (real)2 / d - (real)1;
    }
    smooth(o, W, H, 8, 0, 8, w3, R3, tmp);                                 /* nu3 */
    for (size_t i = 0; i < n; i++) {                                       /* [8 channels, mu] / norm */
        real acc = 0;
        for (int k = 0; k < 8; k++) acc = RFMA(o[i * 8 + k], o[i * 8 + k], acc);
        acc = RFMA(mu, mu, acc);
        real nrm = RSQRT(acc);
        for (int k = 0; k < 8; k++) out[i * 9 + k] = o[i * 8 + k] / nrm;
        out[i * 9 + 8] = mu / nrm;
    }
    free(s); free(o); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Bottom-level correlation (Eq. 3-4)                                         */
/* ------------------------------------------------------------------------- */

/* sim of the atomic patch p (grid index) of I with the 4x4 window of I' at
 * pixel (tx, ty): (1/16) sum over the 16 pixels of the 9-D dot products.
 * Window convention: centre 2 <-> pixels 0..3, i.e. [t-2, t+1]^2;
 * descriptors of I' are zero outside the image, and so are those of the
 * pixels of a partial atomic patch that fall outside I.
 * Order: dx = 0..3 (outer), channel c = 0..8, dy = 0..3 (inner), one fma per
 * term from acc = 0, then one multiplication by 1/16. */
static real corr0(const real* d1, int W1, int H1, const real* d2, int W2, int H2, int px, int py, int tx, int ty) {
    real acc = 0;
    for (int dx = 0; dx < 4; dx++)
        for (int c = 0; c < 9; c++)
            for (int dy = 0; dy < 4; dy++) {
                int x2 = tx - 2 + dx, y2 = ty - 2 + dy;
                int x1 = px - 2 + dx, y1 = py - 2 + dy;
                if (x2 < 0 || y2 < 0 || x2 >= W2 || y2 >= H2) continue;   /* zero term */
                if (x1 >= W1 || y1 >= H1) continue;   /* partial atomic patch: zero term */
                real a = d1[((size_t)y1 * W1 + x1) * 9 + c];
                real b = d2[((size_t)y2 * W2 + x2) * 9 + c];
                acc = RFMA(a, b, acc);
            }
    return acc * (real)0.0625;
}

/* The same C_0 for an atomic patch given as its 144-vector a[(dy*4 + dx)*9 + c]
 * (the pixels of a partial patch outside I already zero: their terms add an
 * exact zero, as the skipped terms of corr0 do): same terms, same order.  The
 * approximate form (Sec. 4.1) passes the prototype that replaces the patch. */
static real corr0_vec(const real* a, const real* d2, int W2, int H2, int tx, int ty) {
    real acc = 0;
    for (int dx = 0; dx < 4; dx++)
        for (int c = 0; c < 9; c++)
            for (int dy = 0; dy < 4; dy++) {
                int x2 = tx - 2 + dx, y2 = ty - 2 + dy;
                if (x2 < 0 || y2 < 0 || x2 >= W2 || y2 >= H2) continue;   /* zero term */
                real b = d2[((size_t)y2 * W2 + x2) * 9 + c];
                acc = RFMA(a[(dy * 4 + dx) * 9 + c], b, acc);
            }
    return acc * (real)0.0625;
}

/* Unpooled, unrectified C_0 for patches [p0, p1): out [p1-p0][H2][W2]. */
int orc_level0(const real* d1, int W1, int H1, const real* d2, int W2, int H2, int p0, int p1, real* out) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = p0; p < p1; p++) {
        int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
        real* o = out + (size_t)(p - p0) * W2 * H2;
        for (int ty = 0; ty < H2; ty++)
            for (int tx = 0; tx < W2; tx++) o[(size_t)ty * W2 + tx] = corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Max-pooling + subsampling (Eq. 8-9) of one map: dst(r) = max over the      */
/* in-domain positions 2r+m, m in {-1,0,1}^2; argmax code (my+1)*3 + (mx+1).  */
/* ------------------------------------------------------------------------- */
/* 3x3 / 2 max-pooling of one map with its argmax; optionally the relative
 * gap (best - second best) / best between the winner and the largest other
 * in-domain candidate of each window (0 on a tie, 1 with a single candidate):
 * how close the argmax decision is to changing. */
static void pool_map(const real* src, int sw, int sh, real* dst, uint8_t* am, double* gap, int dw, int dh,
                     int rectify_after, real lam) {
    for (int ry = 0; ry < dh; ry++)
        for (int rx = 0; rx < dw; rx++) {
            real best = RNEG_INF;
            int code = 4;
            for (int my = -1; my <= 1; my++)
                for (int mx = -1; mx <= 1; mx++) {
                    int x = 2 * rx + mx, y = 2 * ry + my;
                    if (x < 0 || y < 0 || x >= sw || y >= sh) continue;
                    real v = src[(size_t)y * sw + x];
                    if (v > best) { best = v; code = (my + 1) * 3 + (mx + 1); }
                }
            dst[(size_t)ry * dw + rx] = rectify_after ? RPOW(best, lam) : best;
            am[(size_t)ry * dw + rx] = (uint8_t)code;
            if (gap) {
                real second = RNEG_INF;
                for (int my = -1; my <= 1; my++)
                    for (int mx = -1; mx <= 1; mx++) {
                        int x = 2 * rx + mx, y = 2 * ry + my;
                        if (x < 0 || y < 0 || x >= sw || y >= sh || (my + 1) * 3 + (mx + 1) == code) continue;
                        real v = src[(size_t)y * sw + x];
                        if (v > second) second = v;
                    }
                double gp = 1.0;
                if (second != RNEG_INF) gp = best > 0 ? (double)(best - second) / (double)best : 0.0;
                gap[(size_t)ry * dw + rx] = gp;
            }
        }
}

/* Map of one lattice patch at a level >= 1 from its children's pooled maps
 * (Eq. 12): kid[i] = child i's map on the same domain
 * (mw x mh), NULL where child i does not exist; n = number of existing
 * children.  FP64: the rectified average (Algorithm 1 order); FP32 mirror: the
 * unrectified average (the power follows the pooling). */
static void level_average(const real* const* kid, int n, int mw, int mh, int compensated, real lam, real* map) {
    (void)lam;
    (void)compensated;
    for (int qy = 0; qy < mh; qy++)
        for (int qx = 0; qx < mw; qx++) {
#if ORC_F32
            /* FP32 sum over valid children in order i = 0..3: Knuth TwoSum with a
             * running compensation, rounded once at the end (compensated), or one
             * rounding per addition (plain) */
            float s = 0.0f, comp = 0.0f;
#else
            double s = 0.0;
#endif
            for (int i = 0; i < 4; i++) {
                if (!kid[i]) continue;
                int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
                int rx = qx + ox, ry = qy + oy;
                real v = 0;
                if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) v = kid[i][(size_t)ry * mw + rx];
#if ORC_F32
                float t = s + v;
                if (compensated) {
                    float bp = t - s;
                    float err = (s - (t - bp)) + (v - bp);
                    comp = comp + err;
                }
                s = t;
#else
                s += v;
#endif
            }
#if ORC_F32
            map[(size_t)qy * mw + qx] = (s + comp) / (float)n;                 /* rectified after pooling */
#else
            map[(size_t)qy * mw + qx] = RPOW(s / (double)n, lam);
#endif
        }
}

/* ------------------------------------------------------------------------- */
/* The multi-level correlation pyramid (Algorithm 1, Eq. 12, boundary rule)   */
/*                                                                            */
/* pooled[l] : [npatch(l)][dh[l+1]][dw[l+1]]  = (S o P)(C_l), l = 0..L-1      */
/* amax[l]   : same shape, argmax codes                                       */
/* pgap[l]   : same shape, optional (NULL): relative top-two gap of the argmax */
/* top       : [npatch(L)][dh[L]][dw[L]]       = C_L                          */
/* valid[l]  : [npatch(l)] patch membership of G_{4*2^l}, l = 0..L            */
/* cmaps[l]  : optional (NULL, or NULL entries): [npatch(l)][dh[l]][dw[l]],   */
/*             l = 1..L, the level's maps before pooling -- FP64: C_l        */
/*             (rectified); FP32 mirror: the unrectified averages, whose     */
/*             power is C_l                                                    */
/* ------------------------------------------------------------------------- */
static int pyramid_impl(const real* d1, const real* amat, int W1, int H1, const real* d2, int W2, int H2,
                        double lambda, int compensated, real** pooled, uint8_t** amax, real* top, uint8_t** valid,
                        double** pgap, real** cmaps);

int orc_pyramid(const real* d1, int W1, int H1, const real* d2, int W2, int H2, double lambda, int compensated,
                real** pooled, uint8_t** amax, real* top, uint8_t** valid, double** pgap, real** cmaps) {
    return pyramid_impl(d1, NULL, W1, H1, d2, W2, H2, lambda, compensated, pooled, amax, top, valid, pgap, cmaps);
}

/* The pyramid with image 1's atomic patches given as vectors: amat
 * [P0][144] (k = (dy*4 + dx)*9 + c), e.g. each patch replaced by its
 * prototype (approximate form, Sec. 4.1).  W1, H1 fix the geometry. */
int orc_pyramid_vec(const real* amat, int W1, int H1, const real* d2, int W2, int H2, double lambda, int compensated,
                    real** pooled, uint8_t** amax, real* top, uint8_t** valid, double** pgap, real** cmaps) {
    return pyramid_impl(NULL, amat, W1, H1, d2, W2, H2, lambda, compensated, pooled, amax, top, valid, pgap, cmaps);
}

static int pyramid_impl(const real* d1, const real* amat, int W1, int H1, const real* d2, int W2, int H2,
                        double lambda, int compensated, real** pooled, uint8_t** amax, real* top, uint8_t** valid,
                        double** pgap, real** cmaps) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    const real lam = (real)lambda;
    const int L = g.L;

    /* level 0: correlate, rectify, pool (FP64: Algorithm 1 order; FP32: pool then power) */
    int n0 = npatch(&g, 0);
    memset(valid[0], 1, (size_t)n0);
#pragma omp parallel
    {
        real* map = (real*)malloc((size_t)W2 * H2 * sizeof(real));
#pragma omp for schedule(dynamic, 1)
        for (int p = 0; p < n0; p++) {
            int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
            for (int ty = 0; ty < H2; ty++)
                for (int tx = 0; tx < W2; tx++) {
                    real c = amat ? corr0_vec(amat + (size_t)p * 144, d2, W2, H2, tx, ty)
                                  : corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
                    map[(size_t)ty * W2 + tx] = ORC_F32 ? c : RPOW(c, lam);
                }
            size_t off = (size_t)p * g.dw[1] * g.dh[1];
            pool_map(map, W2, H2, pooled[0] + off, amax[0] + off, pgap ? pgap[0] + off : NULL, g.dw[1], g.dh[1],
                     ORC_F32, lam);
        }
        free(map);
    }

    /* levels 1..L: shift-average of the children's pooled maps, rectify, pool */
    for (int l = 1; l <= L; l++) {
        const int np = npatch(&g, l);
        const int mw = g.dw[l], mh = g.dh[l];
        const int cw = g.dw[l], ch = g.dh[l];      /* child pooled maps live on the same domain */
        for (int p = 0; p < np; p++) {
            int any = 0;
            for (int i = 0; i < 4; i++) {
                int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                if (c >= 0 && valid[l - 1][c]) any = 1;
            }
            valid[l][p] = (uint8_t)any;
        }
#pragma omp parallel
        {
            real* map = (real*)malloc((size_t)mw * mh * sizeof(real));
#pragma omp for schedule(dynamic, 1)
            for (int p = 0; p < np; p++) {
                if (!valid[l][p]) continue;
                int ci[4], n = 0;
                for (int i = 0; i < 4; i++) {
                    int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                    ci[i] = (c >= 0 && valid[l - 1][c]) ? c : -1;
                    if (ci[i] >= 0) n++;
                }
                const real* kid[4];
                for (int i = 0; i < 4; i++) kid[i] = ci[i] >= 0 ? pooled[l - 1] + (size_t)ci[i] * cw * ch : NULL;
                level_average(kid, n, mw, mh, compensated, lam, map);
                if (cmaps && cmaps[l]) memcpy(cmaps[l] + (size_t)p * mw * mh, map, (size_t)mw * mh * sizeof(real));
                if (l < L) {
                    size_t off = (size_t)p * g.dw[l + 1] * g.dh[l + 1];
                    pool_map(map, mw, mh, pooled[l] + off, amax[l] + off, pgap ? pgap[l] + off : NULL, g.dw[l + 1],
                             g.dh[l + 1], ORC_F32, lam);
                } else {
                    real* dst = top + (size_t)p * mw * mh;
                    for (size_t k = 0; k < (size_t)mw * mh; k++) dst[k] = ORC_F32 ? RPOW(map[k], lam) : map[k];
                }
            }
            free(map);
        }
    }
    return 0;
}

/* Level-0 pooled maps (same arithmetic as level 0 of orc_pyramid) for a list
 * of atomic patches only: out [n][dh[1]][dw[1]] and argmax codes. */
int orc_level0_pooled(const real* d1, int W1, int H1, const real* d2, int W2, int H2, double lambda,
                      const int* plist, int n, real* out, uint8_t* am) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    const real lam = (real)lambda;
#pragma omp parallel
    {
        real* map = (real*)malloc((size_t)W2 * H2 * sizeof(real));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < n; k++) {
            int p = plist[k];
            int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
            for (int ty = 0; ty < H2; ty++)
                for (int tx = 0; tx < W2; tx++) {
                    real c = corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
                    map[(size_t)ty * W2 + tx] = ORC_F32 ? c : RPOW(c, lam);
                }
            size_t off = (size_t)k * g.dw[1] * g.dh[1];
            pool_map(map, W2, H2, out + off, am + off, NULL, g.dw[1], g.dh[1], ORC_F32, lam);
        }
        free(map);
    }
    return 0;
}

/* Level-1 pooled maps and argmax codes of the listed lattice patches only
 * (same arithmetic as level 1 of orc_pyramid): their children's level-0
 * pooled maps first, then the shifted average, pooling and power.  out
 * [n][dh[2]][dw[2]], am likewise; exists[k] = 0 for a patch with no child
 * (its output is left zero).  For checks of large pairs on sampled patches. */
int orc_level1_pooled(const real* d1, int W1, int H1, const real* d2, int W2, int H2, double lambda, int compensated,
                      const int* plist, int n, real* out, uint8_t* am, uint8_t* exists) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    if (g.L < 2) return -1;
    const real lam = (real)lambda;
    const int mw = g.dw[1], mh = g.dh[1];
    int bad = 0;
#pragma omp parallel
    {
        real* c0 = (real*)malloc((size_t)W2 * H2 * sizeof(real));
        real* kids = (real*)malloc((size_t)4 * mw * mh * sizeof(real));
        uint8_t* kam = (uint8_t*)malloc((size_t)mw * mh);
        real* map = (real*)malloc((size_t)mw * mh * sizeof(real));
        if (!c0 || !kids || !kam || !map) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < n; k++) {
            if (bad) continue;
            const int p = plist[k];
            const real* kid[4];
            int nk = 0;
            for (int i = 0; i < 4; i++) {
                const int c = child_index(&g, 1, p % g.Lx, p / g.Lx, i);
                kid[i] = NULL;
                if (c < 0) continue;
                const int px = 4 * (c % g.P0x) + 2, py = 4 * (c / g.P0x) + 2;
                for (int ty = 0; ty < H2; ty++)
                    for (int tx = 0; tx < W2; tx++) {
                        real v = corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
                        c0[(size_t)ty * W2 + tx] = ORC_F32 ? v : RPOW(v, lam);
                    }
                pool_map(c0, W2, H2, kids + (size_t)i * mw * mh, kam, NULL, mw, mh, ORC_F32, lam);
                kid[i] = kids + (size_t)i * mw * mh;
                nk++;
            }
            exists[k] = (uint8_t)(nk > 0);
            if (!nk) continue;
            level_average(kid, nk, mw, mh, compensated, lam, map);
            const size_t off = (size_t)k * g.dw[2] * g.dh[2];
            pool_map(map, mw, mh, out + off, am + off, NULL, g.dw[2], g.dh[2], ORC_F32, lam);
        }
        free(c0);
        free(kids);
        free(kam);
        free(map);
    }
    return bad ? -2 : 0;
}

/* Existence of every patch at every level (Eq. 7 with the boundary rule of
 * Sec. 3.2): valid[0] = all atomic patches; a lattice patch of level l exists
 * iff one of its children exists.  valid[l]: [npatch(l)], l = 0..L. */
int orc_valid(int W1, int H1, int W2, int H2, uint8_t** valid) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    memset(valid[0], 1, (size_t)npatch(&g, 0));
    for (int l = 1; l <= g.L; l++)
        for (int p = 0; p < npatch(&g, l); p++) {
            int any = 0;
            for (int i = 0; i < 4; i++) {
                int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                if (c >= 0 && valid[l - 1][c]) any = 1;
            }
            valid[l][p] = (uint8_t)any;
        }
    return 0;
}

/* Pooled maps and argmax codes at one level l (0 <= l < L) of the listed
 * patches only, for checks of pairs too large for the whole pyramid: the
 * level-0 maps of their atomic descendants (up to 4^l patches each), then
 * levels 1..l for the descendants only, with the same arithmetic as
 * orc_pyramid (level_average, pool_map).  out [n][dh[l+1]][dw[l+1]], am
 * likewise; exists[k] = valid[l][plist[k]] (a patch that does not exist keeps
 * a zero output). */
int orc_levels_sampled(const real* d1, int W1, int H1, const real* d2, int W2, int H2, double lambda,
                       int compensated, int l, const int* plist, int n, real* out, uint8_t* am, uint8_t* exists) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    if (l < 0 || l >= g.L) return -1;
    const real lam = (real)lambda;
    int rc = 0;
    uint8_t* valid[ORC_MAXL + 1];
    uint8_t* need[ORC_MAXL + 1];
    real** maps[ORC_MAXL + 1];
    for (int k = 0; k <= l; k++) {
        valid[k] = (uint8_t*)calloc((size_t)npatch(&g, k), 1);
        need[k] = (uint8_t*)calloc((size_t)npatch(&g, k), 1);
        maps[k] = (real**)calloc((size_t)npatch(&g, k), sizeof(real*));
        if (!valid[k] || !need[k] || !maps[k]) rc = -2;
    }
    if (rc == 0) {
        /* existence up to level l */
        memset(valid[0], 1, (size_t)npatch(&g, 0));
        for (int k = 1; k <= l; k++)
            for (int p = 0; p < npatch(&g, k); p++) {
                int any = 0;
                for (int i = 0; i < 4; i++) {
                    int c = child_index(&g, k, p % g.Lx, p / g.Lx, i);
                    if (c >= 0 && valid[k - 1][c]) any = 1;
                }
                valid[k][p] = (uint8_t)any;
            }
        /* the descendants the listed patches need, level by level downwards */
        for (int j = 0; j < n; j++) {
            if (plist[j] < 0 || plist[j] >= npatch(&g, l)) { rc = -1; break; }
            exists[j] = valid[l][plist[j]];
            if (exists[j]) need[l][plist[j]] = 1;
        }
        for (int k = l; k >= 1 && rc == 0; k--)
            for (int p = 0; p < npatch(&g, k); p++) {
                if (!need[k][p]) continue;
                for (int i = 0; i < 4; i++) {
                    int c = child_index(&g, k, p % g.Lx, p / g.Lx, i);
                    if (c >= 0 && valid[k - 1][c]) need[k - 1][c] = 1;
                }
            }
    }
    /* level 0: correlate, pool (and rectify) the needed atomic patches */
    if (rc == 0) {
        const int n0 = npatch(&g, 0);
        const size_t sz = (size_t)g.dw[1] * g.dh[1];
        for (int p = 0; p < n0; p++)
            if (need[0][p]) {
                maps[0][p] = (real*)malloc(sz * sizeof(real));
                if (!maps[0][p]) rc = -2;
            }
        if (rc == 0) {
#pragma omp parallel
            {
                real* map = (real*)malloc((size_t)W2 * H2 * sizeof(real));
                uint8_t* am0 = (uint8_t*)malloc(sz);
#pragma omp for schedule(dynamic, 1)
                for (int p = 0; p < n0; p++) {
                    if (!need[0][p] || !map || !am0) continue;
                    int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
                    for (int ty = 0; ty < H2; ty++)
                        for (int tx = 0; tx < W2; tx++) {
                            real c = corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
                            map[(size_t)ty * W2 + tx] = ORC_F32 ? c : RPOW(c, lam);
                        }
                    uint8_t* dst_am = (l == 0) ? NULL : am0;
                    if (l == 0)
                        for (int j = 0; j < n; j++)
                            if (plist[j] == p) dst_am = am + (size_t)j * sz;
                    pool_map(map, W2, H2, maps[0][p], dst_am ? dst_am : am0, NULL, g.dw[1], g.dh[1], ORC_F32, lam);
                }
                if (!map || !am0) {
#pragma omp atomic write
                    rc = -2;
                }
                free(map);
                free(am0);
            }
        }
    }
    /* levels 1..l: shift-average of the children's pooled maps, pool, power */
    for (int k = 1; k <= l && rc == 0; k++) {
        const int mw = g.dw[k], mh = g.dh[k];
        const size_t sz = (size_t)g.dw[k + 1] * g.dh[k + 1];
        for (int p = 0; p < npatch(&g, k); p++)
            if (need[k][p]) {
                maps[k][p] = (real*)malloc(sz * sizeof(real));
                if (!maps[k][p]) rc = -2;
            }
        if (rc) break;
#pragma omp parallel
        {
            real* map = (real*)malloc((size_t)mw * mh * sizeof(real));
            uint8_t* amk = (uint8_t*)malloc(sz);
#pragma omp for schedule(dynamic, 1)
            for (int p = 0; p < npatch(&g, k); p++) {
                if (!need[k][p] || !map || !amk) continue;
                int nk = 0;
                const real* kid[4];
                for (int i = 0; i < 4; i++) {
                    int c = child_index(&g, k, p % g.Lx, p / g.Lx, i);
                    kid[i] = (c >= 0 && valid[k - 1][c]) ? maps[k - 1][c] : NULL;
                    if (kid[i]) nk++;
                }
                level_average(kid, nk, mw, mh, compensated, lam, map);
                uint8_t* dst_am = amk;
                if (k == l)
                    for (int j = 0; j < n; j++)
                        if (plist[j] == p) dst_am = am + (size_t)j * sz;
                pool_map(map, mw, mh, maps[k][p], dst_am, NULL, g.dw[k + 1], g.dh[k + 1], ORC_F32, lam);
            }
            if (!map || !amk) {
#pragma omp atomic write
                rc = -2;
            }
            free(map);
            free(amk);
        }
    }
    if (rc == 0) {
        const size_t sz = (size_t)g.dw[l + 1] * g.dh[l + 1];
        for (int j = 0; j < n; j++)
            if (exists[j]) memcpy(out + (size_t)j * sz, maps[l][plist[j]], sz * sizeof(real));
    }
    for (int k = 0; k <= l; k++) {
        if (maps[k])
            for (int p = 0; p < npatch(&g, k); p++) free(maps[k][p]);
        free(maps[k]);
        free(valid[k]);
        free(need[k]);
    }
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Backtracking with merging (Eq. 13-15) and reciprocal verification (Eq. 16) */
/*                                                                            */
/* The tuple set M starts as every top-level position of every valid patch    */
/* with its score C_L.  One application of B maps each tuple (l, p, q, s) to  */
/* its children (l-1, p_i, t_i = 2(q+o_i)+m_i, s + C_{l-1,p_i}(t_i)); tuples   */
/* equal in (l, p, t) are merged keeping the highest score.  The merged set   */
/* of one level is held in a dense score array (-inf = absent).               */
/* At the atomic level the tuples are reduced on the fly into                */
/*   BestAt(p)   : best tuple of atomic patch p (its own 4x4 cell of I),       */
/*   BestAt'(c)  : best tuple whose t lies in the 4x4 cell c of I'.            */
/* leaf (optional, [P0][H2][W2]): the merged atomic scores themselves.        */
/* leaf_raw (optional, same shape): the same scores unrounded -- the FP32      */
/* mirror's fixed-point integers, exact as doubles -- or -1 where absent.     */
/* reached[l]   : number of distinct tuples at level l (l = 0..L).            */
/* ------------------------------------------------------------------------- */

/* Path scores.  FP64: plain double sums.  FP32 mirror: unsigned
 * fixed point with 28 fractional bits; every term (a map value in [0, 1]) is
 * rounded to the nearest multiple of 2^-28 (ties to even) and the sum of the
 * L + 1 terms (< 16) is exact, hence independent of order and of the merging;
 * it is rounded to FP32 once, at the end. */
#if ORC_F32
typedef uint32_t pscore;
#define PS_NONE 0xFFFFFFFFu
static pscore ps_term(real v) { return (pscore)nearbyintf(v * 268435456.0f); }
static real ps_value(pscore s) { return (real)s * (1.0f / 268435456.0f); }
#else
typedef double pscore;
#define PS_NONE (-INFINITY)
static pscore ps_term(real v) { return v; }
static real ps_value(pscore s) { return s; }
#endif

/* merge: keep the larger score (PS_NONE = absent) */
static int ps_greater(pscore s, pscore cur) { return cur == PS_NONE || s > cur; }

static int better(pscore s, long long idx, pscore bs, long long bidx) {
    return bs == PS_NONE || s > bs || (s == bs && idx < bidx);
}

int orc_backtrack(int W1, int H1, int W2, int H2, real** pooled, uint8_t** amax, const real* top, uint8_t** valid,
                  real* bestP_s, long long* bestP_i, real* bestQ_s, long long* bestQ_i, real* leaf, long long* reached,
                  double** pgap, double* gap, double* leaf_raw) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    const int L = g.L;
    const int n0 = npatch(&g, 0);
    const int CW = (W2 + 3) / 4, CH = (H2 + 3) / 4;
    pscore* bP = (pscore*)malloc((size_t)n0 * sizeof(pscore));
    pscore* bQ = (pscore*)malloc((size_t)CW * CH * sizeof(pscore));
    if (!bP || !bQ) { free(bP); free(bQ); return -2; }
    for (int p = 0; p < n0; p++) { bP[p] = PS_NONE; bestP_i[p] = -1; }
    for (int c = 0; c < CW * CH; c++) { bQ[c] = PS_NONE; bestQ_i[c] = -1; }
    pscore* lf = NULL;
    if (leaf || gap || leaf_raw) {
        lf = (pscore*)malloc((size_t)n0 * W2 * H2 * sizeof(pscore));
        if (!lf) { free(bP); free(bQ); return -2; }
        for (size_t k = 0; k < (size_t)n0 * W2 * H2; k++) lf[k] = PS_NONE;
    }
    /* winning arrival of every merged tuple (decision gaps only): per level l < L,
     * parent flat index at level l + 1 times 4 plus the child index i */
    long long* par[ORC_MAXL + 1];
    for (int l = 0; l <= L; l++) par[l] = NULL;
    if (gap) {
        for (int l = 0; l < L; l++) {
            size_t n = l == 0 ? (size_t)n0 * W2 * H2 : (size_t)npatch(&g, l) * g.dw[l] * g.dh[l];
            par[l] = (long long*)malloc(n * sizeof(long long));
            if (!par[l]) { for (int k = 0; k < l; k++) free(par[k]); free(bP); free(bQ); free(lf); return -2; }
        }
    }
    for (int l = 0; l <= L; l++) reached[l] = 0;

    /* current merged set, level L */
    const int npL = npatch(&g, L);
    size_t ncur = (size_t)npL * g.dw[L] * g.dh[L];
    pscore* cur = (pscore*)malloc(ncur * sizeof(pscore));
    if (!cur) { free(bP); free(bQ); free(lf); return -2; }
    for (int p = 0; p < npL; p++)
        for (size_t k = 0; k < (size_t)g.dw[L] * g.dh[L]; k++) {
            size_t o = (size_t)p * g.dw[L] * g.dh[L] + k;
            cur[o] = valid[L][p] ? ps_term(top[o]) : PS_NONE;
            if (valid[L][p]) reached[L]++;  /* one tuple per (p, q) */
        }

    for (int l = L; l >= 1; l--) {
        const int mw = g.dw[l], mh = g.dh[l];           /* domain of the current level's positions q */
        const int tw = g.dw[l - 1], th = g.dh[l - 1];   /* domain of the children's positions t */
        const int npc = npatch(&g, l - 1);
        pscore* nxt = NULL;
        if (l - 1 >= 1) {
            nxt = (pscore*)malloc((size_t)npc * tw * th * sizeof(pscore));
            if (!nxt) { free(cur); free(bP); free(bQ); free(lf); return -2; }
            for (size_t k = 0; k < (size_t)npc * tw * th; k++) nxt[k] = PS_NONE;
        }
        const int np = npatch(&g, l);
        for (int p = 0; p < np; p++) {
            if (!valid[l][p]) continue;
            for (int qy = 0; qy < mh; qy++)
                for (int qx = 0; qx < mw; qx++) {
                    pscore s = cur[(size_t)p * mw * mh + (size_t)qy * mw + qx];
                    if (s == PS_NONE) continue;
                    for (int i = 0; i < 4; i++) {
                        int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                        if (c < 0 || !valid[l - 1][c]) continue;
                        int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
                        int rx = qx + ox, ry = qy + oy;              /* Eq. 13: 2(q + o_i) + m_i */
                        if (rx < 0 || ry < 0 || rx >= mw || ry >= mh) continue;
                        size_t ro = (size_t)c * mw * mh + (size_t)ry * mw + rx;
                        int code = amax[l - 1][ro];
                        int tx = 2 * rx + (code % 3 - 1), ty = 2 * ry + (code / 3 - 1);
                        pscore s2 = s + ps_term(pooled[l - 1][ro]);   /* Eq. 14: s + C_{N/2,p_i}(p'_i) */
                        const long long arrival = ((long long)p * mw * mh + (long long)qy * mw + qx) * 4 + i;
                        if (l - 1 >= 1) {
                            size_t di = (size_t)c * tw * th + (size_t)ty * tw + tx;
                            pscore* d = &nxt[di];
                            if (ps_greater(s2, *d)) {
                                *d = s2;
                                if (par[l - 1]) par[l - 1][di] = arrival;
                            }
                        } else {
                            long long tidx = (long long)ty * W2 + tx;
                            if (lf) {
                                size_t di = (size_t)c * W2 * H2 + tidx;
                                pscore* d = &lf[di];
                                if (ps_greater(s2, *d)) {
                                    *d = s2;
                                    if (par[0]) par[0][di] = arrival;
                                }
                            }
                            if (better(s2, tidx, bP[c], bestP_i[c])) { bP[c] = s2; bestP_i[c] = tidx; }
                            int cell = (ty / 4) * CW + tx / 4;
                            long long qidx = (long long)c * 16 + (ty % 4) * 4 + (tx % 4);
                            if (better(s2, qidx, bQ[cell], bestQ_i[cell])) { bQ[cell] = s2; bestQ_i[cell] = qidx; }
                        }
                    }
                }
        }
        free(cur);
        cur = nxt;
        if (l - 1 >= 1) {
            long long cnt = 0;
            for (size_t k = 0; k < (size_t)npc * tw * th; k++) cnt += (cur[k] != PS_NONE);
            reached[l - 1] = cnt;
        }
    }
    /* decision gaps (reading of the tolerance rule): for the best tuple of each
     * atomic patch, the smallest relative top-two gap among the decisions that
     * made it the output -- BestAt(p) over the patch's tuples, BestAt' over the
     * tuples of its cell of I', and the 3x3 argmax at every level of the path
     * that merged into it (winning arrival at each level) */
    if (gap) {
        for (int p = 0; p < n0; p++) {
            gap[p] = 1.0;
            if (bestP_i[p] < 0) continue;
            const long long ts = bestP_i[p];
            double g1 = 1.0;
            pscore b1 = bP[p], b2 = PS_NONE;
            for (long long t = 0; t < (long long)W2 * H2; t++) {
                pscore v = lf[(size_t)p * W2 * H2 + t];
                if (t == ts || v == PS_NONE) continue;
                if (b2 == PS_NONE || v > b2) b2 = v;
            }
            if (b2 != PS_NONE) g1 = (double)(ps_value(b1) - ps_value(b2)) / (double)ps_value(b1);
            /* BestAt' of the cell of t */
            const int tx = (int)(ts % W2), ty = (int)(ts / W2);
            pscore c2 = PS_NONE;
            for (int c = 0; c < n0; c++)
                for (int yy = (ty / 4) * 4; yy < (ty / 4) * 4 + 4 && yy < H2; yy++)
                    for (int xx = (tx / 4) * 4; xx < (tx / 4) * 4 + 4 && xx < W2; xx++) {
                        if (c == p && yy == ty && xx == tx) continue;
                        pscore v = lf[(size_t)c * W2 * H2 + (size_t)yy * W2 + xx];
                        if (v == PS_NONE) continue;
                        if (c2 == PS_NONE || v > c2) c2 = v;
                    }
            double g2 = 1.0;
            if (c2 != PS_NONE) g2 = fabs((double)(ps_value(b1) - ps_value(c2))) / (double)ps_value(b1);
            double gm = g1 < g2 ? g1 : g2;
            /* the path: level-m tuple (c, t) came from the level-(m+1) tuple `arrival` via child i,
             * through the argmax of P_m(c, r), r = q + o_i */
            long long idx = (long long)p * W2 * H2 + ts;
            int c = p;
            for (int m = 0; m < L; m++) {
                const long long a = par[m][idx];
                const long long pf = a / 4;
                const int i = (int)(a % 4);
                const int mw = g.dw[m + 1], mh = g.dh[m + 1];
                const int pp = (int)(pf / ((long long)mw * mh));
                const long long q = pf % ((long long)mw * mh);
                const int ox = (i >= 2) ? 1 : -1, oy = (i & 1) ? 1 : -1;
                const int rx = (int)(q % mw) + ox, ry = (int)(q / mw) + oy;
                if (pgap && pgap[m]) {
                    const double d = pgap[m][(size_t)c * mw * mh + (size_t)ry * mw + rx];
                    if (d < gm) gm = d;
                }
                idx = pf;
                c = pp;
            }
            gap[p] = gm;
        }
    }
    for (int l = 0; l <= L; l++) free(par[l]);

    /* scores out, rounded once */
    for (int p = 0; p < n0; p++) bestP_s[p] = bP[p] == PS_NONE ? RNEG_INF : ps_value(bP[p]);
    for (int c = 0; c < CW * CH; c++) bestQ_s[c] = bQ[c] == PS_NONE ? RNEG_INF : ps_value(bQ[c]);
    if (lf) {
        long long cnt = 0;
        for (size_t k = 0; k < (size_t)n0 * W2 * H2; k++) {
            cnt += (lf[k] != PS_NONE);
            if (leaf) leaf[k] = lf[k] == PS_NONE ? RNEG_INF : ps_value(lf[k]);
            if (leaf_raw) leaf_raw[k] = lf[k] == PS_NONE ? -1.0 : (double)lf[k];
        }
        reached[0] = cnt;
    } else {
        reached[0] = -1;   /* not counted without the dense leaf array */
    }
    free(cur);
    free(bP);
    free(bQ);
    free(lf);
    return 0;
}

/* Reciprocal verification (Eq. 16): keep the best tuple of each
 * atomic patch iff it is also the best tuple of its 4x4 cell of I'.  Output in
 * patch order: out[k] = {x1, y1, x2, y2, score}.  Returns the count. */
int orc_reciprocal(int W1, int H1, int W2, int H2, const real* bestP_s, const long long* bestP_i,
                   const real* bestQ_s, const long long* bestQ_i, double* out) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    (void)bestQ_s;
    const int CW = (W2 + 3) / 4;
    int n = 0;
    for (int p = 0; p < g.P0x * g.P0y; p++) {
        if (bestP_i[p] < 0) continue;
        long long t = bestP_i[p];
        int tx = (int)(t % W2), ty = (int)(t / W2);
        int cell = (ty / 4) * CW + tx / 4;
        long long qidx = (long long)p * 16 + (ty % 4) * 4 + (tx % 4);
        if (bestQ_i[cell] != qidx) continue;
        out[5 * n + 0] = 4 * (p % g.P0x) + 2;
        out[5 * n + 1] = 4 * (p / g.P0x) + 2;
        out[5 * n + 2] = tx;
        out[5 * n + 3] = ty;
        out[5 * n + 4] = (double)bestP_s[p];
        n++;
    }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Differentiable form (adjoint of Algorithm 1; the paper has no loss).       */
/* Loss = sum over existing top patches p of max_q C_L(p, q) (first maximum). */
/* Gradients with respect to both descriptor fields, by the chain rule        */
/* through the rectification (Eq. 11), the shifted average (Eq. 12), the      */
/* max-pooling with its argmax (Eq. 9) and the correlation (Eq. 3-4).  Plain  */
/* dense arrays and loops in the forward's order; the unpooled maps of every  */
/* level are kept (small inputs only).                                        */
/* ------------------------------------------------------------------------- */
int orc_loss_grad(const real* d1, int W1, int H1, const real* d2, int W2, int H2, double lambda, double* loss,
                  real* g1, real* g2) {
    geom g;
    if (make_geom(W1, H1, W2, H2, &g)) return -1;
    const real lam = (real)lambda;
    const int L = g.L;
    /* forward, keeping everything: U[l] = unrectified map A_l (l >= 1) or C0 (l = 0)
     * on domain l; P[l] pooled rectified maps on domain l+1 with argmax. */
    real* U[ORC_MAXL + 1];
    real* P[ORC_MAXL];
    uint8_t* M[ORC_MAXL];
    uint8_t* V[ORC_MAXL + 1];
    for (int l = 0; l <= L; l++) {
        U[l] = (real*)calloc((size_t)npatch(&g, l) * g.dw[l] * g.dh[l], sizeof(real));
        V[l] = (uint8_t*)calloc((size_t)npatch(&g, l), 1);
        if (l < L) {
            P[l] = (real*)calloc((size_t)npatch(&g, l) * g.dw[l + 1] * g.dh[l + 1], sizeof(real));
            M[l] = (uint8_t*)calloc((size_t)npatch(&g, l) * g.dw[l + 1] * g.dh[l + 1], 1);
        }
    }
    const int n0 = npatch(&g, 0);
    memset(V[0], 1, (size_t)n0);
    for (int p = 0; p < n0; p++) {
        int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
        for (int ty = 0; ty < H2; ty++)
            for (int tx = 0; tx < W2; tx++) U[0][((size_t)p * H2 + ty) * W2 + tx] = corr0(d1, W1, H1, d2, W2, H2, px, py, tx, ty);
    }
    for (int l = 0; l <= L; l++) {
        const int np = npatch(&g, l), mw = g.dw[l], mh = g.dh[l];
        if (l >= 1) {
            for (int p = 0; p < np; p++) {
                int n = 0;
                for (int i = 0; i < 4; i++) {
                    int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                    if (c >= 0 && V[l - 1][c]) n++;
                }
                V[l][p] = n > 0;
                if (!n) continue;
                for (int qy = 0; qy < mh; qy++)
                    for (int qx = 0; qx < mw; qx++) {
                        real s = 0;
                        for (int i = 0; i < 4; i++) {
                            int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                            if (c < 0 || !V[l - 1][c]) continue;
                            int rx = qx + ((i >= 2) ? 1 : -1), ry = qy + ((i & 1) ? 1 : -1);
                            if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) s += P[l - 1][((size_t)c * mh + ry) * mw + rx];
                        }
                        U[l][((size_t)p * mh + qy) * mw + qx] = s / n;
                    }
            }
        }
        if (l < L) {   /* pool the rectified map */
            const int ow = g.dw[l + 1], oh = g.dh[l + 1];
            for (int p = 0; p < np; p++) {
                if (!V[l][p]) continue;
                for (int ry = 0; ry < oh; ry++)
                    for (int rx = 0; rx < ow; rx++) {
                        real best = RNEG_INF;
                        int code = 4;
                        for (int my = -1; my <= 1; my++)
                            for (int mx = -1; mx <= 1; mx++) {
                                int x = 2 * rx + mx, y = 2 * ry + my;
                                if (x < 0 || y < 0 || x >= mw || y >= mh) continue;
                                real v = RPOW(U[l][((size_t)p * mh + y) * mw + x], lam);
                                if (v > best) { best = v; code = (my + 1) * 3 + (mx + 1); }
                            }
                        P[l][((size_t)p * oh + ry) * ow + rx] = best;
                        M[l][((size_t)p * oh + ry) * ow + rx] = (uint8_t)code;
                    }
            }
        }
    }
    /* adjoints: dU[l] on the unrectified maps */
    real* dU[ORC_MAXL + 1];
    for (int l = 0; l <= L; l++) dU[l] = (real*)calloc((size_t)npatch(&g, l) * g.dw[l] * g.dh[l], sizeof(real));
    double total = 0.0;
    {
        const int np = npatch(&g, L), mw = g.dw[L], mh = g.dh[L];
        for (int p = 0; p < np; p++) {
            if (!V[L][p]) continue;
            real best = RNEG_INF;
            int qb = 0;
            for (int q = 0; q < mw * mh; q++) {
                real v = RPOW(U[L][(size_t)p * mw * mh + q], lam);
                if (v > best) { best = v; qb = q; }
            }
            total += (double)best;
            real u = U[L][(size_t)p * mw * mh + qb];
            dU[L][(size_t)p * mw * mh + qb] = u > 0 ? lam * RPOW(u, lam - 1) : 0;   /* d(u^lam)/du */
        }
    }
    for (int l = L; l >= 1; l--) {
        const int np = npatch(&g, l), mw = g.dw[l], mh = g.dh[l];
        real* dP = (real*)calloc((size_t)npatch(&g, l - 1) * mw * mh, sizeof(real));
        for (int p = 0; p < np; p++) {
            if (!V[l][p]) continue;
            int n = 0;
            for (int i = 0; i < 4; i++) {
                int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                if (c >= 0 && V[l - 1][c]) n++;
            }
            for (int qy = 0; qy < mh; qy++)
                for (int qx = 0; qx < mw; qx++) {
                    real d = dU[l][((size_t)p * mh + qy) * mw + qx];
                    if (d == 0) continue;
                    for (int i = 0; i < 4; i++) {
                        int c = child_index(&g, l, p % g.Lx, p / g.Lx, i);
                        if (c < 0 || !V[l - 1][c]) continue;
                        int rx = qx + ((i >= 2) ? 1 : -1), ry = qy + ((i & 1) ? 1 : -1);
                        if (rx >= 0 && ry >= 0 && rx < mw && ry < mh) dP[((size_t)c * mh + ry) * mw + rx] += d / n;
                    }
                }
        }
        /* pooled value = (U at the argmax)^lam */
        const int cw = g.dw[l - 1], ch = g.dh[l - 1];
        for (int c = 0; c < npatch(&g, l - 1); c++) {
            if (!V[l - 1][c]) continue;
            for (int ry = 0; ry < mh; ry++)
                for (int rx = 0; rx < mw; rx++) {
                    real d = dP[((size_t)c * mh + ry) * mw + rx];
                    if (d == 0) continue;
                    int code = M[l - 1][((size_t)c * mh + ry) * mw + rx];
                    int tx = 2 * rx + code % 3 - 1, ty = 2 * ry + code / 3 - 1;
                    real u = U[l - 1][((size_t)c * ch + ty) * cw + tx];
                    dU[l - 1][((size_t)c * ch + ty) * cw + tx] += u > 0 ? d * lam * RPOW(u, lam - 1) : 0;
                }
        }
        free(dP);
    }
    /* level 0: C0(p, t) = (1/16) sum a_p[k] b_t[k] */
    memset(g1, 0, sizeof(real) * (size_t)W1 * H1 * 9);
    memset(g2, 0, sizeof(real) * (size_t)W2 * H2 * 9);
    for (int p = 0; p < n0; p++) {
        int px = 4 * (p % g.P0x) + 2, py = 4 * (p / g.P0x) + 2;
        for (int ty = 0; ty < H2; ty++)
            for (int tx = 0; tx < W2; tx++) {
                real d = dU[0][((size_t)p * H2 + ty) * W2 + tx];
                if (d == 0) continue;
                d = d / 16;
                for (int dy = 0; dy < 4; dy++)
                    for (int dx = 0; dx < 4; dx++) {
                        int x1 = px - 2 + dx, y1 = py - 2 + dy, x2 = tx - 2 + dx, y2 = ty - 2 + dy;
                        if (x1 >= W1 || y1 >= H1 || x2 < 0 || y2 < 0 || x2 >= W2 || y2 >= H2) continue;
                        for (int c = 0; c < 9; c++) {
                            g1[((size_t)y1 * W1 + x1) * 9 + c] += d * d2[((size_t)y2 * W2 + x2) * 9 + c];
                            g2[((size_t)y2 * W2 + x2) * 9 + c] += d * d1[((size_t)y1 * W1 + x1) * 9 + c];
                        }
                    }
            }
    }
    *loss = total;
    for (int l = 0; l <= L; l++) {
        free(U[l]); free(V[l]); free(dU[l]);
        if (l < L) { free(P[l]); free(M[l]); }
    }
    return 0;
}

/* DeepFlow (Sec. 4.3): the variational refinement that consumes the matches. */
#include "df_oracle.c"
