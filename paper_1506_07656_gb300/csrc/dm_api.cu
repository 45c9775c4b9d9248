// Host side of the C ABI declared in include/dm.h: argument checks,
// geometry, workspace layout, and the launch sequence of each call.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "dm_internal.cuh"

struct dm_ctx {
    dm_config cfg;
    int device;
    DmDescParams desc;
    std::string err;
    // stage timing: DM_NSTAGES + 1 events per recorded call
    std::vector<cudaEvent_t> ev;
    int t_max = 0, t_count = 0;
    long long t_launch0 = 0;
    // autotuner results per pair size (W1, H1, W2, H2)
    std::mutex tune_mu;
    std::map<std::array<int, 4>, DmTune> tuned;
    // batched form: concurrent lanes (internal streams), fork / join events
    int lanes = 2;
    cudaStream_t lane_st[DM_MAX_LANES] = {};
    cudaEvent_t fork_ev = nullptr, join_ev[DM_MAX_LANES] = {};
    // fault injection (dm_inject_fault): test hooks that drive the failure paths
    long long inj_launch = 0;         // > 0: the inj_launch-th next launch site reports a launch failure
    unsigned int inj_table_cap = 0;   // > 0: merge tables of the backtracking capped at this many slots
    long long inj_wait = 0;           // > 0: level-kernel CTAs first wait this many cycles on a barrier nothing completes
    int force_key64 = 0;              // dm_set_merge_keys(64): 64-bit merge keys at every size
    int wave = 1;                     // batched form: pairs per cross-pair wave (dm_set_batch_wave, dm_autotune_batch)
};

// process-wide: > 0, the g_inj_alloc-th next resource creation of the library fails
static std::atomic<long long> g_inj_alloc{0};

namespace {
DmTune tune_for(dm_ctx* c, const DmGeom& g) {
    std::lock_guard<std::mutex> lk(c->tune_mu);
    auto it = c->tuned.find({g.W1, g.H1, g.W2, g.H2});
    return it == c->tuned.end() ? dm_tune_default(g, c->cfg.precision) : it->second;
}
}  // namespace

static std::atomic<long long> g_launches{0};
void dm_count_launches(long long n) { g_launches += n; }
long long dm_launches() { return g_launches.load(); }

namespace {

struct DevGuard {
    int prev = -1;
    bool changed = false;
    explicit DevGuard(int d) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != d) changed = (cudaSetDevice(d) == cudaSuccess);
    }
    ~DevGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

dm_status fail(dm_ctx* c, dm_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

dm_status cuda_fail(dm_ctx* c, cudaError_t e, const char* where) {
    return fail(c, DM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

// Fault injection: true when this launch site is the one dm_inject_fault
// asked to fail (the count runs down over the sites the context reaches).
bool inject_launch(dm_ctx* c) { return c->inj_launch > 0 && --c->inj_launch == 0; }

dm_status injected_launch_failure(dm_ctx* c, const char* where) {
    return fail(c, DM_ECUDA, "%s: injected launch failure", where);
}

// true when this resource creation is the one dm_inject_fault(NULL, DM_FAULT_ALLOC, n) asked to fail
bool inject_alloc() {
    long long v = g_inj_alloc.load();
    while (v > 0)
        if (g_inj_alloc.compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

// The backtracking layout with the merge tables capped by dm_inject_fault
// (at least 64 slots, a multiple of 64, never above the layout's own size).
DmBtLayout capped_tables(const dm_ctx* c, const DmBtLayout& bl) {
    DmBtLayout o = bl;
    if (c->inj_table_cap > 0)
        for (size_t l = 0; l < sizeof(o.cap) / sizeof(o.cap[0]); l++)
            if (o.cap[l] > c->inj_table_cap) o.cap[l] = c->inj_table_cap;
    return o;
}

// Gaussian taps of standard deviation nu on [-ceil(3nu), ceil(3nu)],
// exp(-j^2/(2 nu^2)) in double, normalised by their sum (accumulated from
// j = -R upwards), then rounded to float.  nu <= 0: identity (R = 0).
DmTaps make_taps_d(double nu) {
    DmTaps t;
    memset(&t, 0, sizeof(t));
    if (!(nu > 0.0)) {
        t.R = 0;
        t.w[0] = 1.0f;
        return t;
    }
    int R = (int)ceil(3.0 * nu);
    if (2 * R + 1 > 65) R = 32;
    double v[65], sum = 0.0;
    for (int j = -R; j <= R; j++) {
        v[j + R] = exp(-(double)(j * j) / (2.0 * nu * nu));
        sum += v[j + R];
    }
    for (int j = 0; j <= 2 * R; j++) t.w[j] = (float)(v[j] / sum);
    t.R = R;
    return t;
}

DmTaps make_taps(float nu_f) { return make_taps_d((double)nu_f); }

bool aligned256(const void* p) { return ((uintptr_t)p & 255u) == 0; }

struct MatchLayout {
    DmBtLayout bt;       // at offset 0 (header first)
    size_t desc1, desc2, tmp, img1, img2, out, count, pyr;
    DmPyrLayout py;
    size_t bytes;
};

void match_layout(const DmGeom& g, int precision, MatchLayout* m, bool star = false) {
    dm_bt_layout(g, &m->bt, star);
    size_t o = m->bt.bytes;
    m->desc1 = o; o = dm_align(o + (size_t)g.W1 * g.H1 * 9 * 4);
    m->desc2 = o; o = dm_align(o + (size_t)g.W2 * g.H2 * 9 * 4);
    size_t big = (size_t)g.W1 * g.H1 > (size_t)g.W2 * g.H2 ? (size_t)g.W1 * g.H1 : (size_t)g.W2 * g.H2;
    m->tmp = o; o = dm_align(o + 4 * big * 8 * 4);   // two [H][W][8] buffers per image (both images at once in a wave)
    m->img1 = o; o = dm_align(o + (size_t)g.W1 * g.H1 * 4);
    m->img2 = o; o = dm_align(o + (size_t)g.W2 * g.H2 * 4);
    m->out = o; o = dm_align(o + (size_t)g.npatch(0) * sizeof(dm_match_t));
    m->count = o; o = dm_align(o + 16);
    dm_pyr_layout(g, precision, &m->py);
    m->pyr = o; o = dm_align(o + m->py.bytes);
    m->bytes = o;
}

void fill_pyramid(dm_pyramid* p, const DmGeom& g, int precision, int compensated, const DmTune& tune, const DmPyrLayout& pl,
                  char* base) {
    memset(p, 0, sizeof(*p));
    p->g = g;
    p->precision = precision;
    p->compensated = compensated;
    p->tune = tune;
    for (int l = 0; l <= g.L; l++) p->valid[l] = (const unsigned char*)(base + pl.valid[l]);
    for (int l = 0; l < g.L; l++) {
        p->pooled[l] = (const float*)(base + pl.pooled[l]);
        p->amax[l] = (const unsigned char*)(base + pl.amax[l]);
    }
    p->top = (const float*)(base + pl.top);
    p->proto_of = nullptr;
    p->n0_maps = g.npatch(0);
}

dm_status run_descriptors(dm_ctx* c, const float* img, int W, int H, float* desc, char* tmp, cudaStream_t st) {
    float* a = (float*)tmp;
    float* b = a + (size_t)W * H * 8;
    cudaError_t e = dm_launch_descriptors(c->desc, img, W, H, desc, a, b, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "descriptor kernels");
    return DM_OK;
}

// Pyramid of one pair.  Approximate form (protos != nullptr): level 0 holds
// one map per prototype (n_protos rows of protos) and atomic patch c reads map
// proto_of[c].
dm_status run_pyramid(dm_ctx* c, const DmGeom& g, const float* d1, const float* d2, char* base, const DmPyrLayout& pl,
                      dm_pyramid* py, int* d_status, cudaStream_t st, const float* protos = nullptr, int n_protos = -1,
                      const int* proto_of = nullptr) {
    fill_pyramid(py, g, c->cfg.precision, c->cfg.compensated, tune_for(c, g), pl, base);
    py->inject_wait = c->inj_wait;
    if (protos) {
        py->proto_of = proto_of;
        py->n0_maps = n_protos;
    }
    cudaError_t e;
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(c, e, "clear status");
    if (inject_launch(c)) return injected_launch_failure(c, "level-0 correlation");
    if (c->cfg.precision != DM_FP32) {
        e = dm_launch_corr0_tc(g, c->cfg.precision, d1, d2, c->cfg.lambda, base + pl.a16, d_status,
                               const_cast<float*>(py->pooled[0]), const_cast<unsigned char*>(py->amax[0]),
                               py->tune.m_chunk, st, protos, py->n0_maps);
    } else {
        e = dm_launch_corr0_f32(g, d1, d2, c->cfg.lambda, const_cast<float*>(py->pooled[0]),
                                const_cast<unsigned char*>(py->amax[0]), st, protos, py->n0_maps);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "level-0 correlation");
    if (inject_launch(c)) return injected_launch_failure(c, "pyramid levels");
    e = dm_launch_levels(g, *py, c->cfg.lambda, d_status, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pyramid levels");
    return DM_OK;
}

// Invariant form (Algorithm 2): the transforms whose warped pair the method
// accepts -- a transform that leaves an image too small for one aggregation
// level is skipped -- and the workspace: the call's header, the input pair's
// BestAt / BestAt' arrays, then one dm_match workspace ("region") per lane,
// sized for the largest transform and reused by the transforms of its lane in
// turn (warped images in its image slots).
struct InvLayout {
    size_t header, bestP, bestQ, match, region;
    size_t bytes(int lanes) const { return match + region * (size_t)lanes; }
};

struct InvStep {
    DmInvTransform t;
    DmGeom g;
    MatchLayout ml;
    double cost;          // level-0 products (patches x positions) + a fixed share per transform
};

dm_status inv_plan(dm_ctx* c, const DmGeom& go, std::vector<InvStep>* steps, InvLayout* o) {
    steps->clear();
    size_t mbytes = 0;
    for (int i = 0; i < DM_INV_TRANSFORMS; i++) {
        InvStep s;
        dm_invariant_transform(i, go.W1, go.H1, go.W2, go.H2, &s.t);
        const int r = dm_make_geom(s.t.w1, s.t.h1, s.t.w2, s.t.h2, &s.g);
        if (r == -1) continue;
        if (r != 0)
            return fail(c, DM_EUNSUPPORTED, "invariant form: transform %d (%dx%d / %dx%d) exceeds the supported sizes", i,
                        s.t.w1, s.t.h1, s.t.w2, s.t.h2);
        if (c->force_key64) s.g.key64 = 1;
        match_layout(s.g, c->cfg.precision, &s.ml);
        if (s.ml.bytes > mbytes) mbytes = s.ml.bytes;
        s.cost = (double)s.g.npatch(0) * (double)s.t.w2 * (double)s.t.h2 + 2.0e7;
        steps->push_back(s);
    }
    size_t off = 0;
    o->header = off; off = dm_align(off + sizeof(DmWsHeader));
    o->bestP = off; off = dm_align(off + (size_t)go.npatch(0) * 8);
    o->bestQ = off; off = dm_align(off + (size_t)((go.W2 + 3) / 4) * ((go.H2 + 3) / 4) * 8);
    o->match = off;
    o->region = dm_align(mbytes);
    return DM_OK;
}

// Lane of each transform: longest first, each to the least loaded lane.  The
// results do not depend on it (the reductions into BestAt / BestAt' and the
// header are order-independent).
std::vector<int> inv_schedule(const std::vector<InvStep>& steps, int lanes, std::vector<int>* order) {
    order->resize(steps.size());
    for (size_t i = 0; i < steps.size(); i++) (*order)[i] = (int)i;
    std::sort(order->begin(), order->end(), [&](int a, int b) { return steps[a].cost > steps[b].cost; });
    std::vector<int> lane(steps.size(), 0);
    std::vector<double> load((size_t)lanes, 0.0);
    for (int i : *order) {
        int j = 0;
        for (int k = 1; k < lanes; k++)
            if (load[k] < load[j]) j = k;
        lane[i] = j;
        load[j] += steps[i].cost;
    }
    return lane;
}

dm_status check_geom(dm_ctx* c, int W1, int H1, int W2, int H2, DmGeom* g) {
    int r = dm_make_geom(W1, H1, W2, H2, g);
    if (r == -1) return fail(c, DM_EINVAL, "invalid sizes %dx%d / %dx%d (need W1,H1 >= 4, max(W1,H1) >= 5, W2,H2 >= 1)", W1, H1, W2, H2);
    if (r == -2)
        return fail(c, DM_EUNSUPPORTED, "sizes %dx%d / %dx%d exceed the supported sizes (fixed-point path scores, 32-bit "
                                        "atomic indices)", W1, H1, W2, H2);
    if (c->force_key64) g->key64 = 1;
    return DM_OK;
}

// DM* keeps 32-bit merge keys (its entry lists pack key and score in 64 bits).
dm_status star_keys(dm_ctx* c, const DmGeom& g) {
    if (g.key64)
        return fail(c, DM_EUNSUPPORTED, "DM*: sizes %dx%d / %dx%d need 64-bit merge keys, which DM* does not take", g.W1,
                    g.H1, g.W2, g.H2);
    return DM_OK;
}

}  // namespace

dm_status dm_set_error(dm_ctx* ctx, dm_status s, const char* msg) { return fail(ctx, s, "%s", msg); }
int dm_ctx_device(const dm_ctx* ctx) { return ctx->device; }

// ---------------------------------------------------------------------------
// Geometry and layouts
// ---------------------------------------------------------------------------
// Along one axis of image 1 (n_atomic atomic columns, n_lattice lattice
// columns): does some lattice column hold a patch of level l?  Level-1 column c
// has the atomic children c - 1 and c; level l >= 2 column c the level-(l-1)
// children c - 2^(l-2) and c + 2^(l-2).
static bool dm_axis_level_exists(int n_atomic, int n_lattice, int l) {
    std::vector<char> cur(n_lattice), nxt(n_lattice);
    for (int c = 0; c < n_lattice; c++) cur[c] = (c < n_atomic) || (c >= 1 && c - 1 < n_atomic);
    for (int k = 2; k <= l; k++) {
        const int d = 1 << (k - 2);
        for (int c = 0; c < n_lattice; c++)
            nxt[c] = (c >= d && cur[c - d]) || (c + d < n_lattice && cur[c + d]);
        cur.swap(nxt);
    }
    for (char v : cur)
        if (v) return true;
    return false;
}

int dm_make_geom(int W1, int H1, int W2, int H2, DmGeom* g) {
    memset(g, 0, sizeof(*g));
    if (W1 < 4 || H1 < 4 || W2 < 1 || H2 < 1) return -1;
    if (W1 > (1 << 20) || H1 > (1 << 20) || W2 > (1 << 20) || H2 > (1 << 20)) return -2;
    g->W1 = W1; g->H1 = H1; g->W2 = W2; g->H2 = H2;
    int mx = W1 > H1 ? W1 : H1;
    int L = 0;
    long long N = 4;
    while (N < mx) { N *= 2; L++; }
    if (L < 1) return -1;
    g->P0x = (W1 - 3) / 4 + 1;
    g->P0y = (H1 - 3) / 4 + 1;
    g->Lx = (W1 - 1) / 4 + 1;
    g->Ly = (H1 - 1) / 4 + 1;
    // Algorithm 1 stops at the first N = 4 * 2^L >= max(W1, H1); if image 1 has
    // no patch at that level (a wide, low image whose level-L children all lie
    // 2^L px above and below every lattice point), the pyramid's top is the
    // highest level that has one.  A patch exists iff a child does (Eq. 7 with
    // the boundary rule); the children are two columns times two rows, so a
    // level has a patch iff some column and some row qualify on their own.
    while (L > 1 && !(dm_axis_level_exists(g->P0x, g->Lx, L) && dm_axis_level_exists(g->P0y, g->Ly, L))) L--;
    if (L > DM_MAXL) return -2;
    if (L > 14) return -2;   // fixed-point path scores: L + 1 terms below 2^28 each fit 32 bits
    g->L = L;
    g->dw[0] = W2; g->dh[0] = H2;
    for (int l = 1; l <= L + 1; l++) { g->dw[l] = (g->dw[l - 1] + 1) / 2; g->dh[l] = (g->dh[l - 1] + 1) / 2; }
    // merge keys patch * |domain| + position (levels 1..L-1): 32 bits where they
    // fit, else 64; the atomic indices (pixel of I', patch*16 + offset) must fit 32.
    for (int l = 1; l <= L; l++)
        if ((unsigned long long)g->npatch(l) * (unsigned long long)g->dsize(l) >= 0xffffffffull) g->key64 = 1;
    if ((unsigned long long)g->npatch(0) * 16ull >= 0xffffffffull) return -2;
    if ((unsigned long long)W2 * H2 >= 0xffffffffull) return -2;
    return 0;
}

void dm_pyr_layout(const DmGeom& g, int precision, DmPyrLayout* o) {
    memset(o, 0, sizeof(*o));
    size_t off = 0;
    o->header = off; off = dm_align(off + sizeof(DmWsHeader));
    for (int l = 0; l <= g.L; l++) { o->valid[l] = off; off = dm_align(off + (size_t)g.npatch(l)); }
    for (int l = 0; l < g.L; l++) {
        size_t n = (size_t)g.npatch(l) * (size_t)g.psize(l + 1);
        o->pooled[l] = off; off = dm_align(off + n * 4);
        o->amax[l] = off; off = dm_align(off + n);
    }
    o->top = off; off = dm_align(off + (size_t)g.npatch(g.L) * (size_t)g.dsize(g.L) * 4);
    if (precision != DM_FP32) { o->a16 = off; off = dm_align(off + dm_corr0_tc_a_bytes(g, precision)); }
    o->bytes = off;
}

void dm_bt_layout(const DmGeom& g, DmBtLayout* o, bool star) {
    memset(o, 0, sizeof(*o));
    size_t off = 0;
    o->header = off; off = dm_align(off + sizeof(DmWsHeader));
    // bound on merged tuples per level: B_L = entries; B_l = min(4 B_{l+1}, |P_l|).
    // DM*: level l also receives its local maxima, which are never neighbours,
    // so at most one per 2x2 block of the domain (|P_l| per level, with
    // P_L's size taken as npatch(L) x dsize(L+1)): B_L = that, B_l =
    // min(4 B_{l+1} + |P_l|, 2 |P_l|), and level L has a table too.
    unsigned long long B = (unsigned long long)g.npatch(g.L) * (unsigned long long)g.dsize(g.L);
    const int top = star ? g.L : g.L - 1;
    if (star) B = 0;
    for (int l = top; l >= 1; l--) {
        unsigned long long pooled = (unsigned long long)g.npatch(l) * (unsigned long long)g.dsize(l + 1);
        if (star) B = 4ull * B + pooled < 2ull * pooled ? 4ull * B + pooled : 2ull * pooled;
        else B = 4ull * B < pooled ? 4ull * B : pooled;
        unsigned long long cap = 2ull * B;
        if (cap < 64ull) cap = 64ull;
        if (cap > 0xfffffff0ull) cap = 0xfffffff0ull;
        o->cap[l] = (size_t)cap;
        o->table[l] = off; off = dm_align(off + (size_t)cap * (g.key64 ? 16 : 8));
    }
    o->bestP = off; off = dm_align(off + (size_t)g.npatch(0) * 8);
    o->bestQ = off; off = dm_align(off + (size_t)((g.W2 + 3) / 4) * ((g.H2 + 3) / 4) * 8);
    if (star)
        for (int l = 1; l <= g.L; l++) {     // local maxima: at most one per 2x2 block of the domain
            o->elcap[l] = (size_t)g.npatch(l) * (size_t)g.dsize(l + 1);
            o->elist[l] = off; off = dm_align(off + o->elcap[l] * 8);
        }
    o->bytes = off;
}

size_t dm_desc_tmp_bytes(int W, int H) { return dm_align(2 * (size_t)W * H * 8 * 4); }

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void dm_config_default(dm_config* cfg) {
    if (!cfg) return;
    cfg->nu1 = 1.0f;
    cfg->nu2 = 1.0f;
    cfg->nu3 = 1.0f;
    cfg->slope = 0.2f;
    cfg->mu = 0.3f;
    cfg->lambda = 1.4f;
    cfg->image_scale = 255.0f;
    cfg->precision = DM_FP32;
    cfg->compensated = 1;
}

dm_status dm_create(const dm_config* cfg, int device, dm_ctx** out) {
    if (!out) return DM_EINVAL;
    *out = nullptr;
    dm_config c;
    if (cfg) c = *cfg; else dm_config_default(&c);
    if (!(c.lambda > 0.0f) || !(c.nu1 >= 0.0f) || !(c.nu2 >= 0.0f) || !(c.nu3 >= 0.0f) || !(c.nu1 <= 10.0f) ||
        !(c.nu2 <= 10.0f) || !(c.nu3 <= 10.0f) || !(c.mu >= 0.0f) || !(c.image_scale > 0.0f))
        return DM_EINVAL;
    if (c.precision != DM_FP32 && c.precision != DM_BF16 && c.precision != DM_FP8_E4M3) return DM_EINVAL;
    if (c.compensated != 0 && c.compensated != 1) return DM_EINVAL;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return DM_EINVAL;
    if (inject_alloc()) return DM_ENOMEM;          // fault injection: the context cannot be created
    dm_ctx* x = new (std::nothrow) dm_ctx();
    if (!x) return DM_ENOMEM;
    x->cfg = c;
    x->device = device;
    {
        DevGuard dg(device);
        bool ok = cudaEventCreateWithFlags(&x->fork_ev, cudaEventDisableTiming) == cudaSuccess;
        for (int k = 0; ok && k < DM_MAX_LANES; k++)
            ok = cudaStreamCreateWithFlags(&x->lane_st[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&x->join_ev[k], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            dm_destroy(x);
            return DM_ECUDA;
        }
    }
    x->desc.t1 = make_taps(c.nu1);
    x->desc.t2 = make_taps(c.nu2);
    x->desc.t3 = make_taps(c.nu3);
    x->desc.scale = c.image_scale;
    x->desc.slope = c.slope;
    x->desc.mu = c.mu;
    *out = x;
    return DM_OK;
}

dm_status dm_destroy(dm_ctx* ctx) {
    if (ctx) {
        DevGuard dg(ctx->device);
        for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
        if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
        for (int k = 0; k < DM_MAX_LANES; k++) {
            if (ctx->join_ev[k]) cudaEventDestroy(ctx->join_ev[k]);
            if (ctx->lane_st[k]) cudaStreamDestroy(ctx->lane_st[k]);
        }
    }
    delete ctx;
    return DM_OK;
}

dm_status dm_timing_start(dm_ctx* ctx, int max_calls) {
    if (!ctx || max_calls < 0 || max_calls > 100000) return DM_EINVAL;
    DevGuard dg(ctx->device);
    size_t need = (size_t)max_calls * (DM_NSTAGES + 1);
    while (ctx->ev.size() < need) {
        if (inject_alloc()) return fail(ctx, DM_ENOMEM, "dm_timing_start: injected allocation failure");
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return cuda_fail(ctx, r, "cudaEventCreate");
        ctx->ev.push_back(e);
    }
    ctx->t_max = max_calls;
    ctx->t_count = 0;
    ctx->t_launch0 = dm_launches();
    return DM_OK;
}

dm_status dm_timing_read(dm_ctx* ctx, double* stage_ms, int* n_calls, long long* n_launches) {
    if (!ctx || !stage_ms) return DM_EINVAL;
    DevGuard dg(ctx->device);
    for (int k = 0; k < DM_NSTAGES; k++) stage_ms[k] = 0.0;
    for (int c = 0; c < ctx->t_count; c++) {
        cudaEvent_t* ev = &ctx->ev[(size_t)c * (DM_NSTAGES + 1)];
        cudaError_t r = cudaEventSynchronize(ev[DM_NSTAGES]);
        if (r != cudaSuccess) return cuda_fail(ctx, r, "cudaEventSynchronize");
        for (int k = 0; k < DM_NSTAGES; k++) {
            float ms = 0.f;
            r = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            if (r != cudaSuccess) return cuda_fail(ctx, r, "cudaEventElapsedTime");
            stage_ms[k] += ms;
        }
    }
    if (n_calls) *n_calls = ctx->t_count;
    if (n_launches) *n_launches = dm_launches() - ctx->t_launch0;
    return DM_OK;
}

const char* dm_last_error(const dm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dm_status dm_geometry(int W1, int H1, int W2, int H2, int* L, int* n_patch0, int* n_patch, int* dw, int* dh) {
    DmGeom g;
    int r = dm_make_geom(W1, H1, W2, H2, &g);
    if (r == -1) return DM_EINVAL;
    if (r == -2) return DM_EUNSUPPORTED;
    if (L) *L = g.L;
    if (n_patch0) *n_patch0 = g.npatch(0);
    if (n_patch) *n_patch = g.npatch(1);
    for (int l = 0; l <= g.L + 1; l++) {
        if (dw) dw[l] = g.dw[l];
        if (dh) dh[l] = g.dh[l];
    }
    return DM_OK;
}

dm_status dm_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* desc_bytes,
                             size_t* pyramid_bytes, size_t* backtrack_bytes, size_t* match_bytes) {
    if (!ctx) return DM_EINVAL;
    DmGeom g;
    dm_status s = check_geom(const_cast<dm_ctx*>(ctx), W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    DmPyrLayout pl;
    dm_pyr_layout(g, ctx->cfg.precision, &pl);
    DmBtLayout bl;
    dm_bt_layout(g, &bl);
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml);
    if (desc_bytes) {
        size_t a = dm_desc_tmp_bytes(W1, H1), b = dm_desc_tmp_bytes(W2, H2);
        *desc_bytes = a > b ? a : b;
    }
    if (pyramid_bytes) *pyramid_bytes = pl.bytes;
    if (backtrack_bytes) *backtrack_bytes = bl.bytes;
    if (match_bytes) *match_bytes = ml.bytes;
    return DM_OK;
}

dm_status dm_descriptors(dm_ctx* ctx, const float* d_img, int W, int H, float* d_desc, void* d_tmp, size_t tmp_bytes,
                         void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img || !d_desc || !d_tmp || W < 1 || H < 1) return fail(ctx, DM_EINVAL, "dm_descriptors: bad arguments");
    if (tmp_bytes < dm_desc_tmp_bytes(W, H)) return fail(ctx, DM_ENOMEM, "dm_descriptors: scratch too small");
    DevGuard dg(ctx->device);
    return run_descriptors(ctx, d_img, W, H, d_desc, (char*)d_tmp, (cudaStream_t)stream);
}

dm_status dm_correlate_pyramid(dm_ctx* ctx, const float* d_desc1, int W1, int H1, const float* d_desc2, int W2, int H2,
                               void* d_ws, size_t ws_bytes, dm_pyramid** out, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!out || !d_desc1 || !d_desc2 || !d_ws) return fail(ctx, DM_EINVAL, "dm_correlate_pyramid: null pointer");
    *out = nullptr;
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    DmPyrLayout pl;
    dm_pyr_layout(g, ctx->cfg.precision, &pl);
    if (ws_bytes < pl.bytes) return fail(ctx, DM_ENOMEM, "pyramid workspace %zu < %zu bytes", ws_bytes, pl.bytes);
    DevGuard dg(ctx->device);
    dm_pyramid* py = (dm_pyramid*)malloc(sizeof(dm_pyramid));
    if (!py) return fail(ctx, DM_EINVAL, "host allocation failed");
    DmWsHeader* hdr = reinterpret_cast<DmWsHeader*>((char*)d_ws + pl.header);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(DmWsHeader), (cudaStream_t)stream);   // no backtracking here
    if (e != cudaSuccess) {
        free(py);
        return cuda_fail(ctx, e, "clear header");
    }
    s = run_pyramid(ctx, g, d_desc1, d_desc2, (char*)d_ws, pl, py, &hdr->pyr_status, (cudaStream_t)stream);
    if (s != DM_OK) {
        free(py);
        return s;
    }
    *out = py;
    return DM_OK;
}

dm_status dm_prototypes_workspace_bytes(dm_ctx* ctx, int W1, int H1, int D, size_t* bytes) {
    if (!ctx) return DM_EINVAL;
    if (!bytes) return fail(ctx, DM_EINVAL, "dm_prototypes_workspace_bytes: null pointer");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W1, H1, &g);
    if (s != DM_OK) return s;
    if (D < 1 || D > g.npatch(0)) return fail(ctx, DM_EINVAL, "D = %d outside [1, %d atomic patches]", D, g.npatch(0));
    *bytes = dm_kmeans_ws_bytes(g, D);
    return DM_OK;
}

dm_status dm_prototypes(dm_ctx* ctx, const float* d_desc1, int W1, int H1, int D, int iters, const int* h_init,
                        float* d_protos, int* d_assign, void* d_ws, size_t ws_bytes, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_desc1 || !d_protos || !d_assign || !d_ws || iters < 0) return fail(ctx, DM_EINVAL, "dm_prototypes: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W1, H1, &g);
    if (s != DM_OK) return s;
    const int P0 = g.npatch(0);
    if (D < 1 || D > P0) return fail(ctx, DM_EINVAL, "D = %d outside [1, %d atomic patches]", D, P0);
    const size_t need = dm_kmeans_ws_bytes(g, D);
    if (ws_bytes < need) return fail(ctx, DM_ENOMEM, "prototype workspace %zu < %zu bytes", ws_bytes, need);
    std::vector<int> init(D);
    for (int d = 0; d < D; d++) {
        init[d] = h_init ? h_init[d] : (int)(((long long)d * P0) / D);
        if (init[d] < 0 || init[d] >= P0) return fail(ctx, DM_EINVAL, "init[%d] = %d outside [0, %d)", d, init[d], P0);
    }
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int* d_init = reinterpret_cast<int*>((char*)d_ws + dm_kmeans_init_offset(g, D));
    // a copy from pageable memory returns once the source has been staged, so
    // `init` may go out of scope right after it
    cudaError_t e = cudaMemcpyAsync(d_init, init.data(), (size_t)D * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "copy init");
    e = dm_launch_kmeans(g, d_desc1, D, iters, d_init, d_protos, d_assign, (char*)d_ws, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "k-means kernels");
    return DM_OK;
}

dm_status dm_correlate_pyramid_approx(dm_ctx* ctx, const float* d_protos, int D, const int* d_assign, int W1, int H1,
                                      const float* d_desc2, int W2, int H2, void* d_ws, size_t ws_bytes,
                                      dm_pyramid** out, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!out || !d_protos || !d_assign || !d_desc2 || !d_ws)
        return fail(ctx, DM_EINVAL, "dm_correlate_pyramid_approx: null pointer");
    *out = nullptr;
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    if (D < 1 || D > g.npatch(0)) return fail(ctx, DM_EINVAL, "D = %d outside [1, %d atomic patches]", D, g.npatch(0));
    DmPyrLayout pl;
    dm_pyr_layout(g, ctx->cfg.precision, &pl);
    if (ws_bytes < pl.bytes) return fail(ctx, DM_ENOMEM, "pyramid workspace %zu < %zu bytes", ws_bytes, pl.bytes);
    DevGuard dg(ctx->device);
    dm_pyramid* py = (dm_pyramid*)malloc(sizeof(dm_pyramid));
    if (!py) return fail(ctx, DM_EINVAL, "host allocation failed");
    DmWsHeader* hdr = reinterpret_cast<DmWsHeader*>((char*)d_ws + pl.header);
    cudaError_t e = cudaMemsetAsync(hdr, 0, sizeof(DmWsHeader), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        free(py);
        return cuda_fail(ctx, e, "clear header");
    }
    s = run_pyramid(ctx, g, nullptr, d_desc2, (char*)d_ws, pl, py, &hdr->pyr_status, (cudaStream_t)stream, d_protos, D,
                    d_assign);
    if (s != DM_OK) {
        free(py);
        return s;
    }
    *out = py;
    return DM_OK;
}

dm_status dm_pyramid_level(const dm_pyramid* pyr, int level, const float** d_vals, const unsigned char** d_argmax,
                           const unsigned char** d_valid, int* n_patches, int* mw, int* mh, int* pitch) {
    if (!pyr || level < 0 || level > pyr->g.L) return DM_EINVAL;
    const DmGeom& g = pyr->g;
    if (d_vals) *d_vals = level < g.L ? pyr->pooled[level] : pyr->top;
    if (d_argmax) *d_argmax = level < g.L ? pyr->amax[level] : nullptr;
    if (d_valid) *d_valid = pyr->valid[level];
    if (n_patches) *n_patches = level == 0 ? pyr->n0_maps : g.npatch(level);
    if (mw) *mw = level < g.L ? g.dw[level + 1] : g.dw[level];
    if (mh) *mh = level < g.L ? g.dh[level + 1] : g.dh[level];
    if (pitch) *pitch = level < g.L ? g.pitch(level + 1) : g.dw[level];
    return DM_OK;
}

dm_status dm_pyramid_free(dm_pyramid* pyr) {
    free(pyr);
    return DM_OK;
}

dm_status dm_backtrack(dm_ctx* ctx, const dm_pyramid* pyr, void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity,
                       int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!pyr || !d_ws || !d_out || !d_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_backtrack: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmBtLayout bl;
    dm_bt_layout(pyr->g, &bl);
    if (ws_bytes < bl.bytes) return fail(ctx, DM_ENOMEM, "backtrack workspace %zu < %zu bytes", ws_bytes, bl.bytes);
    DevGuard dg(ctx->device);
    // a stand-alone backtracking workspace carries no pyramid status
    cudaError_t e = cudaMemsetAsync(&reinterpret_cast<DmWsHeader*>((char*)d_ws + bl.header)->pyr_status, 0, sizeof(int),
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clear status");
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "backtracking kernels");
    e = dm_launch_backtrack(pyr->g, *pyr, capped_tables(ctx, bl), (char*)d_ws, d_out, capacity, d_count,
                            (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backtracking kernels");
    return DM_OK;
}

dm_status dm_match(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2, void* d_ws,
                   size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img1 || !d_img2 || !d_ws || !d_out || !d_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_match: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml);
    if (ws_bytes < ml.bytes) return fail(ctx, DM_ENOMEM, "match workspace %zu < %zu bytes", ws_bytes, ml.bytes);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    float* desc1 = (float*)(base + ml.desc1);
    float* desc2 = (float*)(base + ml.desc2);
    cudaEvent_t* ev = nullptr;
    if (ctx->t_count < ctx->t_max) ev = &ctx->ev[(size_t)ctx->t_count++ * (DM_NSTAGES + 1)];
    if (ev) cudaEventRecord(ev[0], st);
    if ((s = run_descriptors(ctx, d_img1, W1, H1, desc1, base + ml.tmp, st)) != DM_OK) return s;
    if ((s = run_descriptors(ctx, d_img2, W2, H2, desc2, base + ml.tmp, st)) != DM_OK) return s;
    if (ev) cudaEventRecord(ev[1], st);
    dm_pyramid py;
    fill_pyramid(&py, g, ctx->cfg.precision, ctx->cfg.compensated, tune_for(ctx, g), ml.py, base + ml.pyr);
    py.inject_wait = ctx->inj_wait;
    cudaError_t e;
    int* d_status = &reinterpret_cast<DmWsHeader*>(base + ml.bt.header)->pyr_status;
    if ((e = cudaMemsetAsync(d_status, 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(ctx, e, "clear status");
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "level-0 correlation");
    if (ctx->cfg.precision != DM_FP32)
        e = dm_launch_corr0_tc(g, ctx->cfg.precision, desc1, desc2, ctx->cfg.lambda, base + ml.pyr + ml.py.a16,
                               d_status, const_cast<float*>(py.pooled[0]), const_cast<unsigned char*>(py.amax[0]),
                               py.tune.m_chunk, st);
    else
        e = dm_launch_corr0_f32(g, desc1, desc2, ctx->cfg.lambda, const_cast<float*>(py.pooled[0]),
                                const_cast<unsigned char*>(py.amax[0]), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "level-0 correlation");
    if (ev) cudaEventRecord(ev[2], st);
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "pyramid levels");
    e = dm_launch_levels(g, py, ctx->cfg.lambda, d_status, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pyramid levels");
    if (ev) cudaEventRecord(ev[3], st);
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "backtracking kernels");
    e = dm_launch_backtrack(g, py, capped_tables(ctx, ml.bt), base, d_out, capacity, d_count, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backtracking kernels");
    if (ev) cudaEventRecord(ev[4], st);
    return DM_OK;
}

dm_status dm_match_host(dm_ctx* ctx, const float* h_img1, int W1, int H1, const float* h_img2, int W2, int H2,
                        void* d_ws, size_t ws_bytes, dm_match_t* h_out, int capacity, int* h_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!h_img1 || !h_img2 || !d_ws || !h_out || !h_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_match_host: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml);
    if (ws_bytes < ml.bytes) return fail(ctx, DM_ENOMEM, "match workspace %zu < %zu bytes", ws_bytes, ml.bytes);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    float* i1 = (float*)(base + ml.img1);
    float* i2 = (float*)(base + ml.img2);
    dm_match_t* dout = (dm_match_t*)(base + ml.out);
    int* dcnt = (int*)(base + ml.count);
    int cap_dev = g.npatch(0);   // at most one match per atomic patch
    cudaError_t e;
    if ((e = cudaMemcpyAsync(i1, h_img1, (size_t)W1 * H1 * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy image 1");
    if ((e = cudaMemcpyAsync(i2, h_img2, (size_t)W2 * H2 * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy image 2");
    if ((s = dm_match(ctx, i1, W1, H1, i2, W2, H2, d_ws, ws_bytes, dout, cap_dev, dcnt, stream)) != DM_OK) return s;
    int ncopy = capacity < cap_dev ? capacity : cap_dev;
    if (ncopy > 0 && (e = cudaMemcpyAsync(h_out, dout, (size_t)ncopy * sizeof(dm_match_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy matches");
    if ((e = cudaMemcpyAsync(h_count, dcnt, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "copy count");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_fail(ctx, e, "dm_match_host");
    if (*h_count > capacity) return fail(ctx, DM_EOVERFLOW, "%d matches, capacity %d", *h_count, capacity);
    return DM_OK;
}

dm_status dm_grad_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* bytes) {
    if (!ctx || !bytes) return DM_EINVAL;
    DmGeom g;
    dm_status s = check_geom(const_cast<dm_ctx*>(ctx), W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    DmGradLayout gl;
    dm_grad_layout(g, &gl);
    if (!gl.cap_ok) return fail(const_cast<dm_ctx*>(ctx), DM_EUNSUPPORTED, "dm_grad_workspace_bytes: gradient frontier above 2^32 entries");
    *bytes = gl.bytes;
    return DM_OK;
}

dm_status dm_loss_grad(dm_ctx* ctx, const dm_pyramid* pyr, const float* d_desc1, const float* d_desc2, void* d_ws,
                       size_t ws_bytes, float* d_loss, float* d_parts, float* d_g1, float* d_g2, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!pyr || !d_desc1 || !d_desc2 || !d_ws || !d_loss) return fail(ctx, DM_EINVAL, "dm_loss_grad: bad arguments");
    if (pyr->proto_of) return fail(ctx, DM_EUNSUPPORTED, "dm_loss_grad: the approximate form has no adjoint");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGradLayout gl;
    dm_grad_layout(pyr->g, &gl);
    if (!gl.cap_ok) return fail(ctx, DM_EUNSUPPORTED, "dm_loss_grad: gradient frontier above 2^32 entries");
    if (ws_bytes < gl.bytes) return fail(ctx, DM_ENOMEM, "gradient workspace %zu < %zu bytes", ws_bytes, gl.bytes);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = dm_launch_loss_grad(pyr->g, *pyr, d_desc1, d_desc2, ctx->cfg.lambda, gl, (char*)d_ws, d_loss, d_g1, d_g2, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gradient kernels");
    if (d_parts) {
        e = cudaMemcpyAsync(d_parts, (char*)d_ws + gl.parts, sizeof(float) * pyr->g.npatch(pyr->g.L), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "copy per-patch maxima");
    }
    return DM_OK;
}

namespace {
// One pair of a wave of the batched form: device images, its workspace slice
// (a match workspace), its output.
struct WavePair {
    const float* img1;
    int W1, H1;
    const float* img2;
    int W2, H2;
    char* base;
    dm_match_t* out;
    int capacity;
    int* count;
};

// A wave of n <= DM_BATCH_MAX pairs in the cross-pair form: every step of the
// method is one launch for all of them (descriptors, the operand packing and
// the level-0 kernel, each level, each step of the backtracking, the
// reciprocal verification) -- the exact form's results, pair by pair.
dm_status run_wave(dm_ctx* ctx, int n, const WavePair* w, cudaStream_t st) {
    DmGeom g[DM_BATCH_MAX];
    MatchLayout ml[DM_BATCH_MAX];
    dm_pyramid py[DM_BATCH_MAX];
    const dm_pyramid* pys[DM_BATCH_MAX];
    DmBtLayout bls[DM_BATCH_MAX];
    const DmBtLayout* blp[DM_BATCH_MAX];
    int* status[DM_BATCH_MAX];
    char* bases[DM_BATCH_MAX];
    dm_match_t* outs[DM_BATCH_MAX];
    int caps[DM_BATCH_MAX];
    int* counts[DM_BATCH_MAX];
    const float* imgs[2 * DM_BATCH_MAX];
    int Ws[2 * DM_BATCH_MAX], Hs[2 * DM_BATCH_MAX];
    float *descs[2 * DM_BATCH_MAX], *tA[2 * DM_BATCH_MAX], *tB[2 * DM_BATCH_MAX];
    const int prec = ctx->cfg.precision;
    cudaError_t e;
    for (int j = 0; j < n; j++) {
        dm_status s = check_geom(ctx, w[j].W1, w[j].H1, w[j].W2, w[j].H2, &g[j]);
        if (s != DM_OK) return s;
        match_layout(g[j], prec, &ml[j]);
        char* base = w[j].base;
        const size_t big = std::max((size_t)g[j].W1 * g[j].H1, (size_t)g[j].W2 * g[j].H2) * 8;
        float* tmp = (float*)(base + ml[j].tmp);
        imgs[2 * j] = w[j].img1;
        Ws[2 * j] = w[j].W1;
        Hs[2 * j] = w[j].H1;
        descs[2 * j] = (float*)(base + ml[j].desc1);
        tA[2 * j] = tmp;
        tB[2 * j] = tmp + big;
        imgs[2 * j + 1] = w[j].img2;
        Ws[2 * j + 1] = w[j].W2;
        Hs[2 * j + 1] = w[j].H2;
        descs[2 * j + 1] = (float*)(base + ml[j].desc2);
        tA[2 * j + 1] = tmp + 2 * big;
        tB[2 * j + 1] = tmp + 3 * big;
        fill_pyramid(&py[j], g[j], prec, ctx->cfg.compensated, tune_for(ctx, g[j]), ml[j].py, base + ml[j].pyr);
        pys[j] = &py[j];
        bls[j] = capped_tables(ctx, ml[j].bt);
        blp[j] = &bls[j];
        status[j] = &reinterpret_cast<DmWsHeader*>(base + ml[j].bt.header)->pyr_status;
        if ((e = cudaMemsetAsync(status[j], 0, sizeof(int), st)) != cudaSuccess) return cuda_fail(ctx, e, "clear status");
        bases[j] = base;
        outs[j] = w[j].out;
        caps[j] = w[j].capacity;
        counts[j] = w[j].count;
    }
    if ((e = dm_launch_descriptors_batch(ctx->desc, 2 * n, imgs, Ws, Hs, descs, tA, tB, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "descriptor kernels");
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "level-0 correlation");
    if (prec != DM_FP32) {
        const float* d1s[DM_BATCH_MAX];
        const float* d2s[DM_BATCH_MAX];
        void* abufs[DM_BATCH_MAX];
        void* sts[DM_BATCH_MAX];
        float* p0[DM_BATCH_MAX];
        unsigned char* a0[DM_BATCH_MAX];
        int mch[DM_BATCH_MAX];
        for (int j = 0; j < n; j++) {
            d1s[j] = descs[2 * j];
            d2s[j] = descs[2 * j + 1];
            abufs[j] = bases[j] + ml[j].pyr + ml[j].py.a16;
            sts[j] = status[j];
            p0[j] = const_cast<float*>(py[j].pooled[0]);
            a0[j] = const_cast<unsigned char*>(py[j].amax[0]);
            mch[j] = py[j].tune.m_chunk;
        }
        e = dm_launch_corr0_tc_batch(n, g, prec, d1s, d2s, ctx->cfg.lambda, abufs, sts, p0, a0, mch, st);
    } else {
        // (the FP32 SIMT kernel runs pair by pair)
        for (int j = 0; j < n && e == cudaSuccess; j++)
            e = dm_launch_corr0_f32(g[j], descs[2 * j], descs[2 * j + 1], ctx->cfg.lambda, const_cast<float*>(py[j].pooled[0]),
                                    const_cast<unsigned char*>(py[j].amax[0]), st);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "level-0 correlation");
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "pyramid levels");
    if ((e = dm_launch_levels_batch(pys, n, ctx->cfg.lambda, status, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "pyramid levels");
    if (inject_launch(ctx)) return injected_launch_failure(ctx, "backtracking kernels");
    if ((e = dm_launch_backtrack_batch(pys, blp, bases, outs, caps, counts, n, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "backtracking kernels");
    return DM_OK;
}

// Waves of the batched form over a workspace of `slices` match workspaces:
// width W (pairs per wave) and lanes K (concurrent waves), K * W <= slices.
void wave_shape(const dm_ctx* ctx, int n, size_t slices, int* W, int* K) {
    int w = std::min(std::min(ctx->wave, n), (int)std::min(slices, (size_t)DM_BATCH_MAX));
    if (w < 1) w = 1;
    const int waves = (n + w - 1) / w;
    int k = (int)std::min(slices / (size_t)w, (size_t)ctx->lanes);
    if (k > waves) k = waves;
    if (k < 1) k = 1;
    *W = w;
    *K = k;
}

// Runs the n pairs of a batch as waves of W pairs on K lanes (fork from and
// join into `st`); wave i covers pairs [i W, i W + W) and runs on lane i % K in
// the slices [lane W, lane W + W) of the workspace.  run(first, count, slice0,
// stream) issues one wave.
extern "C++" template <class F>
dm_status run_waves(dm_ctx* ctx, int n, int W, int K, char* ws, size_t slice, cudaStream_t st, const char* what, F run) {
    const int waves = (n + W - 1) / W;
    if (K == 1) {
        for (int i = 0; i < waves; i++) {
            dm_status s = run(i * W, std::min(W, n - i * W), ws, st);
            if (s != DM_OK) return s;
        }
        return DM_OK;
    }
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    for (int j = 0; e == cudaSuccess && j < K; j++) e = cudaStreamWaitEvent(ctx->lane_st[j], ctx->fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    for (int i = 0; i < waves; i++) {
        const int lane = i % K;
        dm_status s = run(i * W, std::min(W, n - i * W), ws + (size_t)lane * W * slice, ctx->lane_st[lane]);
        if (s != DM_OK) return s;
    }
    for (int j = 0; e == cudaSuccess && j < K; j++) {
        e = cudaEventRecord(ctx->join_ev[j], ctx->lane_st[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[j], 0);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return DM_OK;
}

// workspace of one lane: the largest match workspace over the pairs (256-byte multiple)
dm_status batch_lane_bytes(dm_ctx* ctx, int n, const dm_pair* pairs, size_t* bytes) {
    size_t best = 256;
    for (int k = 0; k < n; k++) {
        size_t mb = 0;
        dm_status s = dm_workspace_bytes(ctx, pairs[k].W1, pairs[k].H1, pairs[k].W2, pairs[k].H2, nullptr, nullptr,
                                         nullptr, &mb);
        if (s != DM_OK) return s;
        if (mb > best) best = mb;
    }
    *bytes = dm_align(best);
    return DM_OK;
}
}  // namespace

dm_status dm_set_merge_keys(dm_ctx* ctx, int bits) {
    if (!ctx) return DM_EINVAL;
    if (bits != 0 && bits != 64) return fail(ctx, DM_EINVAL, "dm_set_merge_keys: bits must be 0 or 64");
    ctx->force_key64 = bits == 64;
    return DM_OK;
}

dm_status dm_set_batch_wave(dm_ctx* ctx, int pairs) {
    if (!ctx) return DM_EINVAL;
    if (pairs < 1 || pairs > DM_BATCH_MAX)
        return fail(ctx, DM_EINVAL, "dm_set_batch_wave: pairs must be in [1, %d]", DM_BATCH_MAX);
    ctx->wave = pairs;
    return DM_OK;
}

dm_status dm_set_batch_lanes(dm_ctx* ctx, int lanes) {
    if (!ctx) return DM_EINVAL;
    if (lanes < 1 || lanes > DM_MAX_LANES) return fail(ctx, DM_EINVAL, "dm_set_batch_lanes: lanes must be 1..%d", DM_MAX_LANES);
    ctx->lanes = lanes;
    return DM_OK;
}

dm_status dm_batch_workspace_bytes(const dm_ctx* ctx, int n, const dm_pair* pairs, size_t* bytes) {
    if (!ctx || n < 0 || (n > 0 && !pairs) || !bytes) return DM_EINVAL;
    size_t lane = 0;
    dm_status s = batch_lane_bytes(const_cast<dm_ctx*>(ctx), n, pairs, &lane);
    if (s != DM_OK) return s;
    const int W = std::max(1, std::min(ctx->wave, n));
    const int waves = n > 0 ? (n + W - 1) / W : 1;
    const int lanes = std::max(1, std::min(ctx->lanes, waves));
    *bytes = lane * (size_t)W * (size_t)lanes;
    return DM_OK;
}

dm_status dm_match_batch(dm_ctx* ctx, int n, const dm_pair* pairs, void* d_ws, size_t ws_bytes, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (n < 0 || (n > 0 && !pairs) || !d_ws) return fail(ctx, DM_EINVAL, "dm_match_batch: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    size_t lane_bytes = 0;
    for (int k = 0; k < n; k++) {     // validate everything before launching anything
        const dm_pair& q = pairs[k];
        if (!q.d_img1 || !q.d_img2 || !q.d_out || !q.d_count || q.capacity < 0)
            return fail(ctx, DM_EINVAL, "dm_match_batch: pair %d: null pointer or negative capacity", k);
        DmGeom g;
        dm_status s = check_geom(ctx, q.W1, q.H1, q.W2, q.H2, &g);
        if (s != DM_OK) return s;
    }
    dm_status s = batch_lane_bytes(ctx, n, pairs, &lane_bytes);
    if (s != DM_OK) return s;
    if (ws_bytes < lane_bytes) return fail(ctx, DM_ENOMEM, "dm_match_batch: needs at least %zu workspace bytes", lane_bytes);
    if (n == 0) return DM_OK;
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int W = 1, K = 1;
    wave_shape(ctx, n, ws_bytes / lane_bytes, &W, &K);
    if (W > 1) {
        return run_waves(ctx, n, W, K, (char*)d_ws, lane_bytes, st, "dm_match_batch: fork / join",
                         [&](int first, int cnt, char* slice0, cudaStream_t ls) -> dm_status {
                             WavePair w[DM_BATCH_MAX];
                             for (int j = 0; j < cnt; j++) {
                                 const dm_pair& q = pairs[first + j];
                                 w[j] = WavePair{q.d_img1, q.W1, q.H1, q.d_img2, q.W2, q.H2, slice0 + (size_t)j * lane_bytes,
                                                 q.d_out, q.capacity, q.d_count};
                             }
                             return run_wave(ctx, cnt, w, ls);
                         });
    }
    int lanes = (int)(ws_bytes / lane_bytes);
    if (lanes > ctx->lanes) lanes = ctx->lanes;
    if (lanes > n) lanes = n;
    if (lanes == 1) {
        for (int k = 0; k < n; k++) {
            const dm_pair& q = pairs[k];
            s = dm_match(ctx, q.d_img1, q.W1, q.H1, q.d_img2, q.W2, q.H2, d_ws, lane_bytes, q.d_out, q.capacity,
                         q.d_count, stream);
            if (s != DM_OK) return s;
        }
        return DM_OK;
    }
    // fork: every lane stream waits for the work already on `stream`; pair k
    // runs on lane k % lanes in its own workspace slice; join back into `stream`
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    for (int j = 0; e == cudaSuccess && j < lanes; j++) e = cudaStreamWaitEvent(ctx->lane_st[j], ctx->fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_batch: fork");
    for (int k = 0; k < n; k++) {
        const dm_pair& q = pairs[k];
        const int j = k % lanes;
        s = dm_match(ctx, q.d_img1, q.W1, q.H1, q.d_img2, q.W2, q.H2, (char*)d_ws + (size_t)j * lane_bytes, lane_bytes,
                     q.d_out, q.capacity, q.d_count, ctx->lane_st[j]);
        if (s != DM_OK) return s;
    }
    for (int j = 0; e == cudaSuccess && j < lanes; j++) {
        e = cudaEventRecord(ctx->join_ev[j], ctx->lane_st[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[j], 0);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_batch: join");
    return DM_OK;
}

namespace {
// One pair of a host-buffer batch on stream `st` in the workspace slice `base`:
// its images copied into the slice's image slots, matched, and the matches and
// the count copied back (all asynchronous).
dm_status run_host_pair(dm_ctx* ctx, const dm_pair_host& q, char* base, size_t bytes, cudaStream_t st) {
    DmGeom g;
    dm_status s = check_geom(ctx, q.W1, q.H1, q.W2, q.H2, &g);
    if (s != DM_OK) return s;
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml);
    float* i1 = (float*)(base + ml.img1);
    float* i2 = (float*)(base + ml.img2);
    dm_match_t* dout = (dm_match_t*)(base + ml.out);
    int* dcnt = (int*)(base + ml.count);
    const int cap_dev = g.npatch(0);   // at most one match per atomic patch
    cudaError_t e;
    if ((e = cudaMemcpyAsync(i1, q.h_img1, (size_t)q.W1 * q.H1 * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "dm_match_batch_host: copy image 1");
    if ((e = cudaMemcpyAsync(i2, q.h_img2, (size_t)q.W2 * q.H2 * 4, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "dm_match_batch_host: copy image 2");
    if ((s = dm_match(ctx, i1, q.W1, q.H1, i2, q.W2, q.H2, base, bytes, dout, cap_dev, dcnt, st)) != DM_OK) return s;
    const int ncopy = q.capacity < cap_dev ? q.capacity : cap_dev;
    if (ncopy > 0 &&
        (e = cudaMemcpyAsync(q.h_out, dout, (size_t)ncopy * sizeof(dm_match_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "dm_match_batch_host: copy matches");
    if ((e = cudaMemcpyAsync(q.h_count, dcnt, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_fail(ctx, e, "dm_match_batch_host: copy count");
    return DM_OK;
}

dm_status batch_host_lane_bytes(dm_ctx* ctx, int n, const dm_pair_host* pairs, size_t* bytes) {
    size_t best = 256;
    for (int k = 0; k < n; k++) {
        size_t mb = 0;
        dm_status s = dm_workspace_bytes(ctx, pairs[k].W1, pairs[k].H1, pairs[k].W2, pairs[k].H2, nullptr, nullptr,
                                         nullptr, &mb);
        if (s != DM_OK) return s;
        if (mb > best) best = mb;
    }
    *bytes = dm_align(best);
    return DM_OK;
}
}  // namespace

dm_status dm_batch_host_workspace_bytes(const dm_ctx* ctx, int n, const dm_pair_host* pairs, size_t* bytes) {
    if (!ctx || n < 0 || (n > 0 && !pairs) || !bytes) return DM_EINVAL;
    size_t lane = 0;
    dm_status s = batch_host_lane_bytes(const_cast<dm_ctx*>(ctx), n, pairs, &lane);
    if (s != DM_OK) return s;
    const int W = std::max(1, std::min(ctx->wave, n));
    const int waves = n > 0 ? (n + W - 1) / W : 1;
    const int lanes = std::max(1, std::min(ctx->lanes, waves));
    *bytes = lane * (size_t)W * (size_t)lanes;
    return DM_OK;
}

dm_status dm_match_batch_host(dm_ctx* ctx, int n, const dm_pair_host* pairs, void* d_ws, size_t ws_bytes, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (n < 0 || (n > 0 && !pairs) || !d_ws) return fail(ctx, DM_EINVAL, "dm_match_batch_host: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    for (int k = 0; k < n; k++) {     // validate everything before copying or launching anything
        const dm_pair_host& q = pairs[k];
        if (!q.h_img1 || !q.h_img2 || !q.h_out || !q.h_count || q.capacity < 0)
            return fail(ctx, DM_EINVAL, "dm_match_batch_host: pair %d: null pointer or negative capacity", k);
        DmGeom g;
        dm_status s = check_geom(ctx, q.W1, q.H1, q.W2, q.H2, &g);
        if (s != DM_OK) return s;
    }
    size_t lane_bytes = 0;
    dm_status s = batch_host_lane_bytes(ctx, n, pairs, &lane_bytes);
    if (s != DM_OK) return s;
    if (ws_bytes < lane_bytes)
        return fail(ctx, DM_ENOMEM, "dm_match_batch_host: needs at least %zu workspace bytes", lane_bytes);
    if (n == 0) return DM_OK;
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int W = 1, K = 1;
    wave_shape(ctx, n, ws_bytes / lane_bytes, &W, &K);
    if (W > 1) {
        return run_waves(ctx, n, W, K, (char*)d_ws, lane_bytes, st, "dm_match_batch_host: fork / join",
                         [&](int first, int cnt, char* slice0, cudaStream_t ls) -> dm_status {
                             WavePair w[DM_BATCH_MAX];
                             MatchLayout ml[DM_BATCH_MAX];
                             cudaError_t e;
                             for (int j = 0; j < cnt; j++) {
                                 const dm_pair_host& q = pairs[first + j];
                                 DmGeom g;
                                 dm_status s2 = check_geom(ctx, q.W1, q.H1, q.W2, q.H2, &g);
                                 if (s2 != DM_OK) return s2;
                                 match_layout(g, ctx->cfg.precision, &ml[j]);
                                 char* base = slice0 + (size_t)j * lane_bytes;
                                 float* i1 = (float*)(base + ml[j].img1);
                                 float* i2 = (float*)(base + ml[j].img2);
                                 if ((e = cudaMemcpyAsync(i1, q.h_img1, (size_t)q.W1 * q.H1 * 4, cudaMemcpyHostToDevice, ls)) !=
                                     cudaSuccess)
                                     return cuda_fail(ctx, e, "dm_match_batch_host: copy image 1");
                                 if ((e = cudaMemcpyAsync(i2, q.h_img2, (size_t)q.W2 * q.H2 * 4, cudaMemcpyHostToDevice, ls)) !=
                                     cudaSuccess)
                                     return cuda_fail(ctx, e, "dm_match_batch_host: copy image 2");
                                 w[j] = WavePair{i1, q.W1, q.H1, i2, q.W2, q.H2, base, (dm_match_t*)(base + ml[j].out),
                                                 g.npatch(0), (int*)(base + ml[j].count)};
                             }
                             dm_status s2 = run_wave(ctx, cnt, w, ls);
                             if (s2 != DM_OK) return s2;
                             for (int j = 0; j < cnt; j++) {
                                 const dm_pair_host& q = pairs[first + j];
                                 const int ncopy = std::min(q.capacity, w[j].capacity);
                                 if (ncopy > 0 && (e = cudaMemcpyAsync(q.h_out, w[j].out, (size_t)ncopy * sizeof(dm_match_t),
                                                                       cudaMemcpyDeviceToHost, ls)) != cudaSuccess)
                                     return cuda_fail(ctx, e, "dm_match_batch_host: copy matches");
                                 if ((e = cudaMemcpyAsync(q.h_count, w[j].count, sizeof(int), cudaMemcpyDeviceToHost, ls)) !=
                                     cudaSuccess)
                                     return cuda_fail(ctx, e, "dm_match_batch_host: copy count");
                             }
                             return DM_OK;
                         });
    }
    int lanes = (int)(ws_bytes / lane_bytes);
    if (lanes > ctx->lanes) lanes = ctx->lanes;
    if (lanes > n) lanes = n;
    if (lanes == 1) {
        for (int k = 0; k < n; k++)
            if ((s = run_host_pair(ctx, pairs[k], (char*)d_ws, lane_bytes, st)) != DM_OK) return s;
        return DM_OK;
    }
    cudaError_t e = cudaEventRecord(ctx->fork_ev, st);
    for (int j = 0; e == cudaSuccess && j < lanes; j++) e = cudaStreamWaitEvent(ctx->lane_st[j], ctx->fork_ev, 0);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_batch_host: fork");
    for (int k = 0; k < n; k++) {
        const int j = k % lanes;
        if ((s = run_host_pair(ctx, pairs[k], (char*)d_ws + (size_t)j * lane_bytes, lane_bytes, ctx->lane_st[j])) != DM_OK)
            return s;
    }
    for (int j = 0; e == cudaSuccess && j < lanes; j++) {
        e = cudaEventRecord(ctx->join_ev[j], ctx->lane_st[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[j], 0);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_batch_host: join");
    return DM_OK;
}

// Autotuner.  Each stage's candidates run back to back on the caller's pair,
// each timed twice with CUDA events (the faster run counts); a candidate
// replaces the current choice only if it is at least 2% faster, so timing
// noise keeps the defaults.
dm_status dm_autotune(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2, void* d_ws,
                      size_t ws_bytes, int* chosen, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img1 || !d_img2 || !d_ws) return fail(ctx, DM_EINVAL, "dm_autotune: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml);
    if (ws_bytes < ml.bytes) return fail(ctx, DM_ENOMEM, "match workspace %zu < %zu bytes", ws_bytes, ml.bytes);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    float* desc1 = (float*)(base + ml.desc1);
    float* desc2 = (float*)(base + ml.desc2);
    if ((s = run_descriptors(ctx, d_img1, W1, H1, desc1, base + ml.tmp, st)) != DM_OK) return s;
    if ((s = run_descriptors(ctx, d_img2, W2, H2, desc2, base + ml.tmp, st)) != DM_OK) return s;
    DmTune best = dm_tune_default(g, ctx->cfg.precision);
    dm_pyramid py;
    fill_pyramid(&py, g, ctx->cfg.precision, ctx->cfg.compensated, best, ml.py, base + ml.pyr);
    int* d_status = &reinterpret_cast<DmWsHeader*>(base + ml.bt.header)->pyr_status;
    dm_match_t* dout = (dm_match_t*)(base + ml.out);
    int* dcnt = (int*)(base + ml.count);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ctx, cudaGetLastError(), "dm_autotune: events");
    }
    cudaError_t err = cudaSuccess;
    // time one run of `stage` (best of three), in ms; < 0 on a CUDA error
    auto timed = [&](auto&& stage) -> float {
        float bestms = -1.0f;
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, st);
            cudaError_t e = stage();
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { err = e; return -1.0f; }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (bestms < 0.0f || ms < bestms) bestms = ms;
        }
        return bestms;
    };
    // a candidate replaces the current shape only when at least 3 % faster (run-to-run
    // differences of a stage are ~1-2 %)
    auto pick = [](float cand, float& cur) { if (cand >= 0.0f && cand < 0.97f * cur) { cur = cand; return true; } return false; };
    cudaMemsetAsync(d_status, 0, sizeof(int), st);
    // level 0: M-tiles per work unit (tensor-core forms only)
    auto level0 = [&]() -> cudaError_t {
        if (ctx->cfg.precision == DM_FP32)
            return dm_launch_corr0_f32(g, desc1, desc2, ctx->cfg.lambda, const_cast<float*>(py.pooled[0]),
                                       const_cast<unsigned char*>(py.amax[0]), st);
        return dm_launch_corr0_tc(g, ctx->cfg.precision, desc1, desc2, ctx->cfg.lambda, base + ml.pyr + ml.py.a16, d_status,
                                  const_cast<float*>(py.pooled[0]), const_cast<unsigned char*>(py.amax[0]),
                                  py.tune.m_chunk, st);
    };
    // one untimed run first: the default shape is timed warm like the candidates after it
    if ((err = level0()) != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(ctx, err, "dm_autotune");
    }
    float cur = timed(level0);
    if (ctx->cfg.precision != DM_FP32) {
        const int n_mtiles = (g.npatch(0) + 127) / 128;
        const int splits[] = {1, 2, 3, 4, 6, 8};
        for (int k : splits) {
            const int mc = (n_mtiles + k - 1) / k;
            if (mc == best.m_chunk) continue;   // the default, timed above
            py.tune.m_chunk = mc;
            if (pick(timed(level0), cur)) best.m_chunk = mc;
        }
        py.tune.m_chunk = best.m_chunk;
    }
    // levels: pooled rows per CTA tile x ring columns
    auto levels = [&]() { return dm_launch_levels(g, py, ctx->cfg.lambda, d_status, st); };
    levels();
    cur = timed(levels);
    // rows per tile x ring (the default first, timed above); 0 = row-streaming kernel
    const int lshapes[6][2] = {{16, 2}, {16, 3}, {8, 3}, {4, 2}, {4, 3}, {0, 2}};
    for (const auto& sh : lshapes) {
        py.tune.level_th = sh[0];
        py.tune.level_ring = sh[1];
        if (pick(timed(levels), cur)) { best.level_th = sh[0]; best.level_ring = sh[1]; }
    }
    py.tune.level_th = best.level_th;
    py.tune.level_ring = best.level_ring;
    // backtracking: CTAs per SM of the expansion kernels
    auto backtrack = [&]() { return dm_launch_backtrack(g, py, ml.bt, base, dout, g.npatch(0), dcnt, st); };
    backtrack();
    cur = timed(backtrack);
    const int mults[] = {2, 4, 16, 32};
    for (int m : mults) {
        py.tune.bt_mult = m;
        if (pick(timed(backtrack), cur)) best.bt_mult = m;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "dm_autotune");
    DmWsHeader h;
    if ((err = cudaMemcpy(&h, base + ml.bt.header, sizeof(h), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, err, "dm_autotune: status");
    if (h.pyr_status || h.status) return fail(ctx, DM_ETIMEOUT, "dm_autotune: device status %d / %d", h.pyr_status, h.status);
    {
        std::lock_guard<std::mutex> lk(ctx->tune_mu);
        ctx->tuned[{W1, H1, W2, H2}] = best;
    }
    if (chosen) { chosen[0] = best.m_chunk; chosen[1] = best.level_th; chosen[2] = best.bt_mult; chosen[3] = best.level_ring; }
    return DM_OK;
}

dm_status dm_autotune_batch(dm_ctx* ctx, int n, const dm_pair* pairs, void* d_ws, size_t ws_bytes, int* chosen,
                            void* stream) {
    if (!ctx) return DM_EINVAL;
    if (n < 1 || !pairs || !d_ws) return fail(ctx, DM_EINVAL, "dm_autotune_batch: bad arguments");
    size_t lane = 0;
    dm_status s = batch_lane_bytes(ctx, n, pairs, &lane);
    if (s != DM_OK) return s;
    const size_t slices = ws_bytes / lane;
    if (slices < 1) return fail(ctx, DM_ENOMEM, "dm_autotune_batch: needs at least %zu workspace bytes", lane);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int wave0 = ctx->wave, lanes0 = ctx->lanes;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(ctx, cudaGetLastError(), "dm_autotune_batch: events");
    }
    // (wave width, lanes) within the workspace: each pair on its own launches
    // on 1..4 lanes, and waves of 2..8 pairs on 1..4 lanes
    int best_w = 1, best_k = 1;
    float best_ms = -1.0f;
    dm_status rs = DM_OK;
    for (int w : {1, 2, 3, 4, 6, 8}) {
        if (w > n || (size_t)w > slices || w > DM_BATCH_MAX) continue;
        const int waves = (n + w - 1) / w;
        for (int k = 1; k <= DM_MAX_LANES; k++) {
            if ((size_t)(w * k) > slices || k > waves) break;
            ctx->wave = w;
            ctx->lanes = k;
            float ms = -1.0f;
            // one untimed run (one-time set-up), then the best of two
            rs = dm_match_batch(ctx, n, pairs, d_ws, (size_t)w * k * lane, st);
            for (int r = 0; r < 2 && rs == DM_OK; r++) {
                cudaEventRecord(e0, st);
                rs = dm_match_batch(ctx, n, pairs, d_ws, (size_t)w * k * lane, st);
                cudaEventRecord(e1, st);
                float t = -1.0f;
                if (rs == DM_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
                if (t >= 0.0f && (ms < 0.0f || t < ms)) ms = t;
            }
            if (rs != DM_OK) break;
            if (ms >= 0.0f && (best_ms < 0.0f || ms < 0.98f * best_ms)) {
                best_ms = ms;
                best_w = w;
                best_k = k;
            }
        }
        if (rs != DM_OK) break;
    }
    // then, in that shape, the CTAs per SM of the backtracking expansions for all the
    // batch's pair sizes together: concurrent lanes share the SMs, so the grid
    // that is best for a pair alone need not be best here
    if (rs == DM_OK) {
        ctx->wave = best_w;
        ctx->lanes = best_k;
        std::vector<std::array<int, 4>> sizes;
        for (int j = 0; j < n; j++) {
            const std::array<int, 4> key{pairs[j].W1, pairs[j].H1, pairs[j].W2, pairs[j].H2};
            if (std::find(sizes.begin(), sizes.end(), key) == sizes.end()) sizes.push_back(key);
        }
        std::vector<DmTune> tunes0;
        for (const auto& key : sizes) {
            DmGeom g;
            dm_make_geom(key[0], key[1], key[2], key[3], &g);
            tunes0.push_back(tune_for(ctx, g));
        }
        auto set_mult = [&](int m) {
            std::lock_guard<std::mutex> lk(ctx->tune_mu);
            for (size_t i = 0; i < sizes.size(); i++) {
                DmTune t = tunes0[i];
                if (m > 0) t.bt_mult = m;
                ctx->tuned[sizes[i]] = t;
            }
        };
        int best_m = 0;                      // 0: each size keeps its own
        for (int m : {4, 8, 16}) {
            set_mult(m);
            float ms = -1.0f;
            rs = dm_match_batch(ctx, n, pairs, d_ws, (size_t)best_w * best_k * lane, st);
            for (int r = 0; r < 2 && rs == DM_OK; r++) {
                cudaEventRecord(e0, st);
                rs = dm_match_batch(ctx, n, pairs, d_ws, (size_t)best_w * best_k * lane, st);
                cudaEventRecord(e1, st);
                float t = -1.0f;
                if (rs == DM_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
                if (t >= 0.0f && (ms < 0.0f || t < ms)) ms = t;
            }
            if (rs != DM_OK) break;
            if (ms >= 0.0f && ms < 0.98f * best_ms) {
                best_ms = ms;
                best_m = m;
            }
        }
        set_mult(best_m);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rs != DM_OK) {
        ctx->wave = wave0;
        ctx->lanes = lanes0;
        return rs;
    }
    ctx->wave = best_w;
    ctx->lanes = best_k;
    if (chosen) {
        chosen[0] = best_w;
        chosen[1] = best_k;
    }
    return DM_OK;
}

dm_status dm_tuned_config(dm_ctx* ctx, int W1, int H1, int W2, int H2, int* chosen) {
    if (!ctx || !chosen) return DM_EINVAL;
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    const DmTune t = tune_for(ctx, g);
    chosen[0] = t.m_chunk;
    chosen[1] = t.level_th;
    chosen[2] = t.bt_mult;
    chosen[3] = t.level_ring;
    return DM_OK;
}

dm_status dm_set_tuned_config(dm_ctx* ctx, int W1, int H1, int W2, int H2, const int* chosen) {
    if (!ctx || !chosen) return DM_EINVAL;
    if (chosen[0] < 1 || (chosen[1] != 0 && chosen[1] != 4 && chosen[1] != 8 && chosen[1] != 16) || chosen[2] < 1 ||
        chosen[2] > 64 ||
        (chosen[3] != 2 && chosen[3] != 3))
        return fail(ctx, DM_EINVAL, "dm_set_tuned_config: invalid launch shapes %d %d %d %d", chosen[0], chosen[1],
                    chosen[2], chosen[3]);
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s != DM_OK) return s;
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned[{W1, H1, W2, H2}] = DmTune{chosen[0], chosen[1], chosen[2], chosen[3]};
    return DM_OK;
}

// ---------------------------------------------------------------------------
// DeepFlow (Sec. 4.3)
// ---------------------------------------------------------------------------
void dm_flow_params_default(dm_flow_params* p) {
    if (!p) return;
    p->sigma = 0.5; p->eta = 0.95; p->gamma = 0.8; p->delta = 0.0; p->beta = 300.0; p->b = 0.6; p->kappa = 5.0;
    p->zeta = 0.1; p->eps = 0.001; p->sigma_m = 50.0; p->omega = 1.6; p->image_scale = 255.0;
    p->n_fixed = 5; p->n_sor = 25; p->min_size = 16;
}

namespace {
dm_status flow_check(dm_ctx* ctx, int W, int H, int capacity, const dm_flow_params* prm, dm_flow_params* q) {
    if (prm) *q = *prm;
    else dm_flow_params_default(q);
    if (W < 1 || H < 1 || capacity < 0) return fail(ctx, DM_EINVAL, "DeepFlow: bad size %dx%d or capacity %d", W, H, capacity);
    if ((long long)W * H > (1LL << 30)) return fail(ctx, DM_EUNSUPPORTED, "DeepFlow: %dx%d is too large", W, H);
    if (!(q->eta > 0.0 && q->eta < 1.0) || q->min_size < 1 || q->n_fixed < 0 || q->n_sor < 0 || !(q->eps > 0.0) ||
        !(q->sigma_m > 0.0) || !(q->omega > 0.0 && q->omega < 2.0) || !(q->sigma >= 0.0) || !(q->image_scale > 0.0))
        return fail(ctx, DM_EINVAL, "DeepFlow: parameter out of range");
    return DM_OK;
}
}  // namespace

dm_status dm_deepflow_workspace_bytes(dm_ctx* ctx, int W, int H, int capacity, const dm_flow_params* prm, size_t* bytes) {
    if (!ctx) return DM_EINVAL;
    if (!bytes) return fail(ctx, DM_EINVAL, "dm_deepflow_workspace_bytes: bytes is NULL");
    dm_flow_params q;
    dm_status s = flow_check(ctx, W, H, capacity, prm, &q);
    if (s != DM_OK) return s;
    DmFlowPlan plan;
    dm_flow_plan(W, H, capacity, q, &plan);
    *bytes = plan.bytes;
    return DM_OK;
}

dm_status dm_deepflow(dm_ctx* ctx, const float* d_img1, const float* d_img2, int W, int H, const dm_match_t* d_matches,
                      const int* d_count, int capacity, const dm_flow_params* prm, float* d_u, float* d_v, void* d_ws,
                      size_t ws_bytes, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img1 || !d_img2 || !d_u || !d_v || !d_ws) return fail(ctx, DM_EINVAL, "dm_deepflow: bad arguments");
    if ((d_matches == nullptr) != (d_count == nullptr))
        return fail(ctx, DM_EINVAL, "dm_deepflow: give both d_matches and d_count, or neither");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    dm_flow_params q;
    dm_status s = flow_check(ctx, W, H, d_matches ? capacity : 0, prm, &q);
    if (s != DM_OK) return s;
    DmFlowPlan plan;
    dm_flow_plan(W, H, d_matches ? capacity : 0, q, &plan);
    if (ws_bytes < plan.bytes) return fail(ctx, DM_ENOMEM, "DeepFlow workspace %zu < %zu bytes", ws_bytes, plan.bytes);
    DevGuard dg(ctx->device);
    const DmTaps taps = make_taps_d(q.sigma);
    cudaError_t e = dm_launch_deepflow(plan, taps, d_img1, d_img2, d_matches, d_count, d_u, d_v, (char*)d_ws,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DeepFlow kernels");
    return DM_OK;
}

// ---------------------------------------------------------------------------
// DM* (Sec. 5.3): local-maximum entry points at every level, start + end scores
// ---------------------------------------------------------------------------
dm_status dm_star_workspace_bytes(const dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* backtrack_bytes,
                                  size_t* match_bytes) {
    if (!ctx) return DM_EINVAL;
    DmGeom g;
    dm_status s = check_geom(const_cast<dm_ctx*>(ctx), W1, H1, W2, H2, &g);
    if (s == DM_OK) s = star_keys(const_cast<dm_ctx*>(ctx), g);
    if (s != DM_OK) return s;
    DmBtLayout bl;
    dm_bt_layout(g, &bl, true);
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml, true);
    if (backtrack_bytes) *backtrack_bytes = bl.bytes;
    if (match_bytes) *match_bytes = ml.bytes;
    return DM_OK;
}

dm_status dm_backtrack_star(dm_ctx* ctx, const dm_pyramid* pyr, void* d_ws, size_t ws_bytes, dm_match_t* d_out,
                            int capacity, int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!pyr || !d_ws || !d_out || !d_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_backtrack_star: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    dm_status s = star_keys(ctx, pyr->g);
    if (s != DM_OK) return s;
    DmBtLayout bl;
    dm_bt_layout(pyr->g, &bl, true);
    if (ws_bytes < bl.bytes) return fail(ctx, DM_ENOMEM, "DM* backtrack workspace %zu < %zu bytes", ws_bytes, bl.bytes);
    DevGuard dg(ctx->device);
    cudaError_t e = cudaMemsetAsync(&reinterpret_cast<DmWsHeader*>((char*)d_ws + bl.header)->pyr_status, 0, sizeof(int),
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "clear status");
    e = dm_launch_backtrack_star(pyr->g, *pyr, bl, (char*)d_ws, ctx->cfg.lambda, d_out, capacity, d_count,
                                 (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DM* backtracking kernels");
    return DM_OK;
}

dm_status dm_match_star(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                        void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img1 || !d_img2 || !d_ws || !d_out || !d_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_match_star: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom g;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &g);
    if (s == DM_OK) s = star_keys(ctx, g);
    if (s != DM_OK) return s;
    MatchLayout ml;
    match_layout(g, ctx->cfg.precision, &ml, true);
    if (ws_bytes < ml.bytes) return fail(ctx, DM_ENOMEM, "DM* match workspace %zu < %zu bytes", ws_bytes, ml.bytes);
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    float* desc1 = (float*)(base + ml.desc1);
    float* desc2 = (float*)(base + ml.desc2);
    if ((s = run_descriptors(ctx, d_img1, W1, H1, desc1, base + ml.tmp, st)) != DM_OK) return s;
    if ((s = run_descriptors(ctx, d_img2, W2, H2, desc2, base + ml.tmp, st)) != DM_OK) return s;
    dm_pyramid py;
    int* d_status = &reinterpret_cast<DmWsHeader*>(base + ml.bt.header)->pyr_status;
    if ((s = run_pyramid(ctx, g, desc1, desc2, base + ml.pyr, ml.py, &py, d_status, st)) != DM_OK) return s;
    cudaError_t e = dm_launch_backtrack_star(g, py, ml.bt, base, ctx->cfg.lambda, d_out, capacity, d_count, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "DM* backtracking kernels");
    return DM_OK;
}

// ---------------------------------------------------------------------------
// Scale and rotation invariant form (Sec. 4.2, Algorithm 2)
// ---------------------------------------------------------------------------
dm_status dm_invariant_workspace_bytes(dm_ctx* ctx, int W1, int H1, int W2, int H2, size_t* bytes) {
    if (!ctx) return DM_EINVAL;
    if (!bytes) return fail(ctx, DM_EINVAL, "dm_invariant_workspace_bytes: bytes is NULL");
    DmGeom go;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &go);
    if (s != DM_OK) return s;
    std::vector<InvStep> steps;
    InvLayout il;
    if ((s = inv_plan(ctx, go, &steps, &il)) != DM_OK) return s;
    const int lanes = (int)steps.size() < ctx->lanes ? (int)steps.size() : ctx->lanes;
    *bytes = il.bytes(lanes > 0 ? lanes : 1);
    return DM_OK;
}

dm_status dm_match_invariant(dm_ctx* ctx, const float* d_img1, int W1, int H1, const float* d_img2, int W2, int H2,
                             void* d_ws, size_t ws_bytes, dm_match_t* d_out, int capacity, int* d_count, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_img1 || !d_img2 || !d_ws || !d_out || !d_count || capacity < 0)
        return fail(ctx, DM_EINVAL, "dm_match_invariant: bad arguments");
    if (!aligned256(d_ws)) return fail(ctx, DM_EINVAL, "workspace must be 256-byte aligned");
    DmGeom go;
    dm_status s = check_geom(ctx, W1, H1, W2, H2, &go);
    if (s != DM_OK) return s;
    std::vector<InvStep> steps;
    InvLayout il;
    if ((s = inv_plan(ctx, go, &steps, &il)) != DM_OK) return s;
    if (ws_bytes < il.bytes(1)) return fail(ctx, DM_ENOMEM, "invariant workspace %zu < %zu bytes", ws_bytes, il.bytes(1));
    // lanes: the context's count, as many as the workspace holds, at most one per transform
    int lanes = ctx->lanes < (int)steps.size() ? ctx->lanes : (int)steps.size();
    while (lanes > 1 && ws_bytes < il.bytes(lanes)) lanes--;
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)d_ws;
    DmWsHeader* hdr = reinterpret_cast<DmWsHeader*>(base + il.header);
    unsigned long long* bestP = reinterpret_cast<unsigned long long*>(base + il.bestP);
    unsigned long long* bestQ = reinterpret_cast<unsigned long long*>(base + il.bestQ);
    cudaError_t e;
    if ((e = cudaMemsetAsync(hdr, 0, sizeof(DmWsHeader), st)) != cudaSuccess) return cuda_fail(ctx, e, "clear header");
    if ((e = cudaMemsetAsync(bestP, 0, il.bestQ - il.bestP, st)) != cudaSuccess) return cuda_fail(ctx, e, "clear BestAt");
    if ((e = cudaMemsetAsync(bestQ, 0, il.match - il.bestQ, st)) != cudaSuccess) return cuda_fail(ctx, e, "clear BestAt'");
    std::vector<int> order;
    const std::vector<int> lane_of = inv_schedule(steps, lanes, &order);
    // fork: with several lanes every lane stream waits for the work already on `stream`
    if (lanes > 1) {
        e = cudaEventRecord(ctx->fork_ev, st);
        for (int j = 0; e == cudaSuccess && j < lanes; j++) e = cudaStreamWaitEvent(ctx->lane_st[j], ctx->fork_ev, 0);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_invariant: fork");
    }
    for (int i : order) {
        const InvStep& sp = steps[i];
        const DmInvTransform& t = sp.t;
        const MatchLayout& ml = sp.ml;
        const int j = lane_of[i];
        cudaStream_t ls = lanes > 1 ? ctx->lane_st[j] : st;
        char* mb = base + il.match + il.region * (size_t)j;
        float* w1 = (float*)(mb + ml.img1);
        float* w2 = (float*)(mb + ml.img2);
        DmRect rect;
        rect.t1 = dm_make_xform(W1, H1, t.w1, t.h1, t.s1, 0);
        rect.t2 = dm_make_xform(W2, H2, t.w2, t.h2, t.s2, t.k);
        rect.W1 = W1; rect.H1 = H1; rect.W2 = W2; rect.H2 = H2;
        rect.P0x = go.P0x; rect.P0y = go.P0y;
        rect.bestP = bestP;
        rect.bestQ = bestQ;
        if ((e = dm_launch_warp(d_img1, W1, H1, w1, t.w1, t.h1, rect.t1, ls)) != cudaSuccess) return cuda_fail(ctx, e, "warp");
        if ((e = dm_launch_warp(d_img2, W2, H2, w2, t.w2, t.h2, rect.t2, ls)) != cudaSuccess) return cuda_fail(ctx, e, "warp");
        float* desc1 = (float*)(mb + ml.desc1);
        float* desc2 = (float*)(mb + ml.desc2);
        if ((s = run_descriptors(ctx, w1, t.w1, t.h1, desc1, mb + ml.tmp, ls)) != DM_OK) return s;
        if ((s = run_descriptors(ctx, w2, t.w2, t.h2, desc2, mb + ml.tmp, ls)) != DM_OK) return s;
        DmWsHeader* th = reinterpret_cast<DmWsHeader*>(mb + ml.bt.header);
        dm_pyramid py;
        if ((s = run_pyramid(ctx, sp.g, desc1, desc2, mb + ml.pyr, ml.py, &py, &th->pyr_status, ls)) != DM_OK) return s;
        e = dm_launch_backtrack(sp.g, py, ml.bt, mb, nullptr, 0, nullptr, ls, &rect);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "backtracking kernels");
        if ((e = dm_launch_inv_fold(hdr, th, ls)) != cudaSuccess) return cuda_fail(ctx, e, "status fold");
    }
    if (lanes > 1) {
        for (int j = 0; e == cudaSuccess && j < lanes; j++) {
            e = cudaEventRecord(ctx->join_ev[j], ctx->lane_st[j]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->join_ev[j], 0);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_match_invariant: join");
    }
    e = dm_launch_reciprocal(go, bestP, bestQ, hdr, d_out, capacity, d_count, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "reciprocal verification");
    return DM_OK;
}

dm_status dm_inject_fault(dm_ctx* ctx, int kind, long long arg) {
    if (arg < 0) return fail(ctx, DM_EINVAL, "dm_inject_fault: negative argument");
    if (kind == DM_FAULT_ALLOC) {
        g_inj_alloc.store(arg);
        return DM_OK;
    }
    if (!ctx) return DM_EINVAL;
    switch (kind) {
        case DM_FAULT_NONE:
            ctx->inj_launch = 0;
            ctx->inj_table_cap = 0;
            ctx->inj_wait = 0;
            g_inj_alloc.store(0);
            return DM_OK;
        case DM_FAULT_LAUNCH:
            ctx->inj_launch = arg;
            return DM_OK;
        case DM_FAULT_CAPACITY:
            if (arg > 0xffffffffLL) return fail(ctx, DM_EINVAL, "dm_inject_fault: capacity too large");
            // whole blocks of 64 slots (the hashing keeps blocks of 32 keys together)
            ctx->inj_table_cap = arg == 0 ? 0u : (unsigned int)(((arg + 63) / 64) * 64);
            return DM_OK;
        case DM_FAULT_WAIT:
            ctx->inj_wait = arg;
            return DM_OK;
        default:
            return fail(ctx, DM_EINVAL, "dm_inject_fault: unknown kind %d", kind);
    }
}

dm_status dm_read_status(dm_ctx* ctx, const void* d_ws, int* status, long long* reached, int n_reached, void* stream) {
    if (!ctx) return DM_EINVAL;
    if (!d_ws || !status || n_reached < 0 || n_reached > DM_MAXL + 2) return fail(ctx, DM_EINVAL, "dm_read_status: bad arguments");
    DevGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    DmWsHeader h;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d_ws, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "dm_read_status");
    *status = h.status | (h.pyr_status ? DM_DEV_TIMEOUT : 0);
    for (int l = 0; l < n_reached && reached; l++) reached[l] = (long long)h.count[l];
    return DM_OK;
}

}  // extern "C"
