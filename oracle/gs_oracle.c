/*
 * gs_oracle.c -- plain, slow FP64 CPU oracle of the anchor-Gaussian rendering
 * path (decode -> project -> bin/sort -> composite -> L1 -> reverse pass).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two only see the same
 * seeded inputs.
 *
 * Every step is written out in the order of the method, one element at a
 * time, in double precision, with no blocking, fusion or reordering:
 *   - anchor visibility and per-anchor decoding: Sec. III-A (Eq. 2) and the
 *     partitioned decoder of Sec. III-D (Eq. 6), following the Scaffold-GS
 *     anchor representation the paper adopts;
 *   - projection of each 3D Gaussian to a 2D conic (Sec. III-A, 3DGS
 *     preliminaries) with the EWA constants of the 3DGS rasterizer the paper
 *     builds on;
 *   - tile binning with (tile, depth) keys and a sort on (key, splat id);
 *   - front-to-back alpha compositing, Eq. 1;
 *   - the L1 photometric term of Eq. 3 and its structural (SSIM) term;
 *   - the optimizer step (Adam) and the densification statistics;
 *   - map maintenance: voxelisation (Eq. 4) and the loop-closure
 *     deformation (Eq. 7);
 *   - the analytic reverse pass of all of the above (the method is
 *     "differentiable", Sec. II/III-A), derived by hand from the forward
 *     definitions and checked against central finite differences.
 *
 * Readings of points the paper leaves open (all shared with the GPU path by
 * specification, not by code): near plane 0.2, visibility margin 15 % of the
 * image per side, low-pass 0.3 px^2, tangent clamp 1.3, radius
 * ceil(3 sqrt(lambda_max)) with eigen-floor 0.1, alpha clamp 0.99, skip
 * alpha < 1/255, stop when T' < 1e-4 (the crossing splat is not composited),
 * pixel (u,v) sampled at integer coordinates, 16x16 tiles, ties ordered by
 * splat id.
 *
 * Camera record: double[16] = fx, fy, cx, cy, R[9] (row-major world->camera),
 * t[3]; resolution int[2] = width, height.
 */
#include <limits.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_TILE 16
static const double O_NEAR = 0.2;
static const double O_MARGIN = 0.15;
static const double O_LOWPASS = 0.3;
static const double O_TANCLAMP = 1.3;
static const double O_ALPHA_MAX = 0.99;
static const double O_ALPHA_MIN = 1.0 / 255.0;
static const double O_T_MIN = 1e-4;

typedef struct {
    double fx, fy, cx, cy, R[9], t[3];
    int W, H, TX, TY;
    long tile_base, pix_base;
} ocam;

static void load_cams(int V, const double *cams, const int *wh, ocam *out)
{
    long tb = 0, pb = 0;
    for (int v = 0; v < V; ++v) {
        const double *c = cams + 16 * v;
        ocam *o = out + v;
        o->fx = c[0]; o->fy = c[1]; o->cx = c[2]; o->cy = c[3];
        for (int i = 0; i < 9; ++i) o->R[i] = c[4 + i];
        for (int i = 0; i < 3; ++i) o->t[i] = c[13 + i];
        o->W = wh[2 * v]; o->H = wh[2 * v + 1];
        o->TX = (o->W + O_TILE - 1) / O_TILE;
        o->TY = (o->H + O_TILE - 1) / O_TILE;
        o->tile_base = tb; o->pix_base = pb;
        tb += (long)o->TX * o->TY;
        pb += (long)o->W * o->H;
    }
}

/* world point -> camera coordinates p = R x + t */
static void to_cam(const ocam *c, const double x[3], double p[3])
{
    for (int i = 0; i < 3; ++i)
        p[i] = c->R[3 * i] * x[0] + c->R[3 * i + 1] * x[1] + c->R[3 * i + 2] * x[2] + c->t[i];
}

/* camera centre x_c = -R^T t */
static void cam_centre(const ocam *c, double xc[3])
{
    for (int i = 0; i < 3; ++i)
        xc[i] = -(c->R[i] * c->t[0] + c->R[3 + i] * c->t[1] + c->R[6 + i] * c->t[2]);
}

static int near_rel(double x, double thr, double band)
{
    return fabs(x - thr) <= band * fabs(thr);
}

/* FNV-1a over 64-bit words: a fingerprint of every discrete decision. */
static void fnv(uint64_t *h, uint64_t w)
{
    for (int i = 0; i < 8; ++i) {
        *h ^= (w >> (8 * i)) & 0xff;
        *h *= 1099511628211ULL;
    }
}

/* ------------------------------------------------------------------------ */
/* a0: anchor visibility.  An anchor is decoded for a view iff its centre is
 * in front of the near plane and projects inside the image grown by 15 % per
 * side.  Rows are emitted view-major, in anchor order.  Returns the number of
 * rows, or -(rows) when that exceeds `cap` (nothing past cap is written). */
long gso_visibility(int N, const double *xyz, int V, const double *cams, const int *wh,
                    double band, int *av_anchor, long *view_start, long cap,
                    unsigned char *row_flag)
{
    ocam *cs = (ocam *)malloc(sizeof(ocam) * (V > 0 ? V : 1));
    load_cams(V, cams, wh, cs);
    long r = 0;
    for (int v = 0; v < V; ++v) {
        const ocam *c = cs + v;
        view_start[v] = r;
        double lox = -O_MARGIN * c->W, hix = (1.0 + O_MARGIN) * c->W;
        double loy = -O_MARGIN * c->H, hiy = (1.0 + O_MARGIN) * c->H;
        for (int a = 0; a < N; ++a) {
            double p[3];
            to_cam(c, xyz + 3 * a, p);
            int flag = near_rel(p[2], O_NEAR, band);
            if (!(p[2] > O_NEAR)) continue;
            double u = c->fx * p[0] / p[2] + c->cx;
            double w = c->fy * p[1] / p[2] + c->cy;
            if (!(u >= lox && u < hix && w >= loy && w < hiy)) continue;
            flag |= fabs(u - lox) <= band * (fabs(lox) + 1) || fabs(u - hix) <= band * hix ||
                    fabs(w - loy) <= band * (fabs(loy) + 1) || fabs(w - hiy) <= band * hiy;
            if (r < cap) {
                av_anchor[r] = a;
                if (row_flag) row_flag[r] = (unsigned char)flag;
            }
            ++r;
        }
    }
    view_start[V] = r;
    free(cs);
    return r <= cap ? r : -r;
}

/* ------------------------------------------------------------------------ */
/* a1: decode of one (view, anchor) row with its partition's MLP set (Eq. 6).
 * Input u = [f_a, d_ac, delta_ac] (Eq. 2); three heads z_h = W2 relu(W1 u +
 * b1) + b2 with outputs (k, 3k, 7k).  Activations: opacity = tanh, colour =
 * sigmoid, scale = exp(l[3:6]) * sigmoid, rotation = normalised quaternion
 * (w,x,y,z); position mu = x_a + offset * exp(l[0:3]). */

typedef struct {
    const double *W1, *b1, *W2, *b2;
    int din, dout;
} ohead;

static void head_ptrs(const double *mlp_m, int F, int k, int Hd, ohead h[3])
{
    int din = F + 4;
    int douts[3] = {k, 3 * k, 7 * k};
    const double *p = mlp_m;
    for (int i = 0; i < 3; ++i) {
        h[i].din = din; h[i].dout = douts[i];
        h[i].W1 = p; p += (long)Hd * din;
        h[i].b1 = p; p += Hd;
        h[i].W2 = p; p += (long)douts[i] * Hd;
        h[i].b2 = p; p += douts[i];
    }
}

static long mlp_size(int F, int k, int Hd)
{
    long din = F + 4, s = 0;
    int douts[3] = {k, 3 * k, 7 * k};
    for (int i = 0; i < 3; ++i) s += Hd * din + Hd + (long)douts[i] * Hd + douts[i];
    return s;
}

static double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

/* builds u, runs the three heads; pre/hid: [3][Hd]; z: [3][7k] */
static void mlp_forward(const ohead h[3], int Hd, const double *u, double *pre, double *hid,
                        double *z, int zstride)
{
    for (int hh = 0; hh < 3; ++hh) {
        for (int j = 0; j < Hd; ++j) {
            double s = h[hh].b1[j];
            for (int i = 0; i < h[hh].din; ++i) s += h[hh].W1[(long)j * h[hh].din + i] * u[i];
            pre[hh * Hd + j] = s;
            hid[hh * Hd + j] = s > 0.0 ? s : 0.0;
        }
        for (int o = 0; o < h[hh].dout; ++o) {
            double s = h[hh].b2[o];
            for (int j = 0; j < Hd; ++j) s += h[hh].W2[(long)o * Hd + j] * hid[hh * Hd + j];
            z[hh * zstride + o] = s;
        }
    }
}

static void make_input(const double *xa, const double *fa, int F, const double xc[3], double *u,
                       double d[3], double *delta)
{
    for (int i = 0; i < 3; ++i) d[i] = xa[i] - xc[i];
    double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    *delta = n;
    for (int i = 0; i < F; ++i) u[i] = fa[i];
    for (int i = 0; i < 3; ++i) u[F + i] = d[i] / n;
    u[F + 3] = n;
}

int gso_decode(int N, int F, int k, int Hd, int M, const double *xyz, const double *feat,
               const double *log_scaling, const double *offsets, const int *part,
               const double *mlp, int V, const double *cams, const int *wh, long rows,
               const int *av_anchor, const long *view_start, double band, double *mu,
               double *scale, double *quat, double *opacity, double *colour,
               unsigned char *cand_flag)
{
    (void)N; (void)M;
    ocam *cs = (ocam *)malloc(sizeof(ocam) * V);
    load_cams(V, cams, wh, cs);
    long msz = mlp_size(F, k, Hd);
    int din = F + 4;
    double *u = (double *)malloc(sizeof(double) * din);
    double *pre = (double *)malloc(sizeof(double) * 3 * Hd);
    double *hid = (double *)malloc(sizeof(double) * 3 * Hd);
    double *z = (double *)malloc(sizeof(double) * 3 * 7 * k);
    for (int v = 0; v < V; ++v) {
        double xc[3];
        cam_centre(cs + v, xc);
        for (long r = view_start[v]; r < view_start[v + 1]; ++r) {
            int a = av_anchor[r];
            ohead h[3];
            head_ptrs(mlp + (long)part[a] * msz, F, k, Hd, h);
            double d[3], delta;
            make_input(xyz + 3 * a, feat + (long)a * F, F, xc, u, d, &delta);
            mlp_forward(h, Hd, u, pre, hid, z, 7 * k);
            const double *ls = log_scaling + 6 * a;
            for (int i = 0; i < k; ++i) {
                long c = r * k + i;
                double zo = z[i];
                opacity[c] = tanh(zo);
                if (cand_flag) cand_flag[c] = fabs(zo) <= band;
                for (int ch = 0; ch < 3; ++ch) colour[3 * c + ch] = sigm(z[7 * k + 3 * i + ch]);
                for (int j = 0; j < 3; ++j)
                    scale[3 * c + j] = exp(ls[3 + j]) * sigm(z[14 * k + 7 * i + j]);
                const double *qz = z + 14 * k + 7 * i + 3;
                double qn = sqrt(qz[0] * qz[0] + qz[1] * qz[1] + qz[2] * qz[2] + qz[3] * qz[3]);
                for (int j = 0; j < 4; ++j) quat[4 * c + j] = qz[j] / qn;
                const double *off = offsets + ((long)a * k + i) * 3;
                for (int j = 0; j < 3; ++j) mu[3 * c + j] = xyz[3 * a + j] + off[j] * exp(ls[j]);
            }
        }
    }
    free(u); free(pre); free(hid); free(z); free(cs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a2: projection of one 3D Gaussian (EWA splatting).  Sigma3 = Rq S^2 Rq^T;
 * J from the perspective map with x/z, y/z clamped to +-1.3 half-FOV;
 * Sigma2 = J R Sigma3 R^T J^T + 0.3 I; conic = Sigma2^-1; radius
 * ceil(3 sqrt(lambda_max)); tile rectangle [x0,x1) x [y0,y1). */

static void quat_to_rot(const double q[4], double Rq[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    Rq[0] = 1 - 2 * (y * y + z * z); Rq[1] = 2 * (x * y - w * z);     Rq[2] = 2 * (x * z + w * y);
    Rq[3] = 2 * (x * y + w * z);     Rq[4] = 1 - 2 * (x * x + z * z); Rq[5] = 2 * (y * z - w * x);
    Rq[6] = 2 * (x * z - w * y);     Rq[7] = 2 * (y * z + w * x);     Rq[8] = 1 - 2 * (x * x + y * y);
}

static long view_of(long c, int k, int V, const long *view_start)
{
    long r = c / k;
    for (int v = 0; v < V; ++v)
        if (r < view_start[v + 1]) return v;
    return V - 1;
}

/* The rectangle decisions floor((m +- r)/16) and ceil(3 sqrt(lambda)) depend
 * on values FP32 knows to a few ulp, so their band is 1/20 of the others. */
static int near_int_edge(double x, double band)
{
    band *= 0.05;
    /* x close to an integer (a floor/ceil decision that FP32 may flip) */
    double f = x - floor(x);
    return f <= band * (fabs(x) + 1.0) || (1.0 - f) <= band * (fabs(x) + 1.0);
}

/* status[c]: 0 culled, 1 valid splat (may still cover no tile) */
int gso_project(long C, int k, int V, const long *view_start, const double *cams, const int *wh,
                const double *mu, const double *scale, const double *quat,
                const double *opacity, double band, double *mean2d, double *conic,
                double *cov2d, double *depth, int *rect, int *tiles, int *status,
                unsigned char *flag, int *fp64_branch)
{
    ocam *cs = (ocam *)malloc(sizeof(ocam) * V);
    load_cams(V, cams, wh, cs);
    for (long c = 0; c < C; ++c) {
        const ocam *cm = cs + view_of(c, k, V, view_start);
        int fl = 0;
        status[c] = 0; tiles[c] = 0;
        rect[4 * c] = rect[4 * c + 1] = rect[4 * c + 2] = rect[4 * c + 3] = 0;
        mean2d[2 * c] = mean2d[2 * c + 1] = 0;
        conic[3 * c] = conic[3 * c + 1] = conic[3 * c + 2] = 0;
        cov2d[3 * c] = cov2d[3 * c + 1] = cov2d[3 * c + 2] = 0;
        depth[c] = 0;
        if (fp64_branch) fp64_branch[c] = 0;
        if (flag) flag[c] = 0;
        if (!(opacity[c] > 0.0)) continue;
        double p[3];
        to_cam(cm, mu + 3 * c, p);
        fl |= near_rel(p[2], O_NEAR, band);   /* bit 0: the splat's presence may flip */
        if (!(p[2] > O_NEAR)) { if (flag) flag[c] = (unsigned char)fl; continue; }
        /* Sigma3 = Rq diag(s^2) Rq^T */
        double Rq[9], S3[9];
        quat_to_rot(quat + 4 * c, Rq);
        const double *s = scale + 3 * c;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += Rq[3 * i + l] * s[l] * s[l] * Rq[3 * j + l];
                S3[3 * i + j] = acc;
            }
        /* Jacobian of the perspective map at the (clamped) point */
        double limx = O_TANCLAMP * (cm->W / (2.0 * cm->fx));
        double limy = O_TANCLAMP * (cm->H / (2.0 * cm->fy));
        double txz = p[0] / p[2], tyz = p[1] / p[2];
        txz = txz < -limx ? -limx : (txz > limx ? limx : txz);
        tyz = tyz < -limy ? -limy : (tyz > limy ? limy : tyz);
        double J[6] = {cm->fx / p[2], 0.0, -cm->fx * txz / p[2],
                       0.0, cm->fy / p[2], -cm->fy * tyz / p[2]};
        double T[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[3 * i + j] = J[3 * i] * cm->R[j] + J[3 * i + 1] * cm->R[3 + j] +
                               J[3 * i + 2] * cm->R[6 + j];
        double S2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l)
                    for (int m = 0; m < 3; ++m) acc += T[3 * i + l] * S3[3 * l + m] * T[3 * j + m];
                S2[2 * i + j] = acc;
            }
        double a = S2[0] + O_LOWPASS, b = S2[1], cc = S2[3] + O_LOWPASS;
        cov2d[3 * c] = a; cov2d[3 * c + 1] = b; cov2d[3 * c + 2] = cc;
        double det = a * cc - b * b;
        if (fp64_branch) fp64_branch[c] = det < 1e-3 * a * cc;
        fl |= det <= band * a * cc;
        if (!(det > 0.0)) { if (flag) flag[c] = (unsigned char)fl; continue; }
        conic[3 * c] = cc / det;
        conic[3 * c + 1] = -b / det;
        conic[3 * c + 2] = a / det;
        double mid = 0.5 * (a + cc);
        double disc = mid * mid - det;
        double lam = mid + sqrt(disc > 0.1 ? disc : 0.1);
        double r3 = 3.0 * sqrt(lam);
        double r = ceil(r3);
        fl |= near_int_edge(r3, band) << 1;   /* bit 1: the tile rectangle may flip */
        double mx = cm->fx * p[0] / p[2] + cm->cx;
        double my = cm->fy * p[1] / p[2] + cm->cy;
        mean2d[2 * c] = mx; mean2d[2 * c + 1] = my;
        depth[c] = p[2];
        double ex[4] = {(mx - r) / O_TILE, (mx + r) / O_TILE, (my - r) / O_TILE, (my + r) / O_TILE};
        for (int i = 0; i < 4; ++i) fl |= near_int_edge(ex[i], band) << 1;
        long x0 = (long)floor(ex[0]), x1 = (long)floor(ex[1]) + 1;
        long y0 = (long)floor(ex[2]), y1 = (long)floor(ex[3]) + 1;
        x0 = x0 < 0 ? 0 : (x0 > cm->TX ? cm->TX : x0);
        x1 = x1 < 0 ? 0 : (x1 > cm->TX ? cm->TX : x1);
        y0 = y0 < 0 ? 0 : (y0 > cm->TY ? cm->TY : y0);
        y1 = y1 < 0 ? 0 : (y1 > cm->TY ? cm->TY : y1);
        rect[4 * c] = (int)x0; rect[4 * c + 1] = (int)y0;
        rect[4 * c + 2] = (int)x1; rect[4 * c + 3] = (int)y1;
        tiles[c] = (int)((x1 - x0) * (y1 - y0));
        status[c] = 1;
        if (flag) flag[c] = (unsigned char)fl;
    }
    free(cs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a3: binning and sort.  Each splat emits one key per covered tile:
 * key = (global tile id << 32) | bits(float32 depth); value = splat id.
 * Pairs are sorted on (key, value) -- a total order, so the result is
 * unique -- and each global tile gets its [start, end) range. */

typedef struct { uint64_t key; uint32_t val; } opair;

static int pair_cmp(const void *pa, const void *pb)
{
    const opair *a = (const opair *)pa, *b = (const opair *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

long gso_bin_sort(long C, int k, int V, const long *view_start, const int *wh,
                  const uint32_t *depth_bits, const int *rect, long cap, uint64_t *keys,
                  uint32_t *vals, uint32_t *ranges)
{
    ocam *cs = (ocam *)calloc(V, sizeof(ocam));
    double *zc = (double *)calloc(16 * (size_t)V, sizeof(double));
    load_cams(V, zc, wh, cs);
    long P = 0;
    for (long c = 0; c < C; ++c)
        P += (long)(rect[4 * c + 2] - rect[4 * c]) * (rect[4 * c + 3] - rect[4 * c + 1]);
    long Ttot = cs[V - 1].tile_base + (long)cs[V - 1].TX * cs[V - 1].TY;
    for (long t = 0; t < 2 * Ttot; ++t) ranges[t] = 0;
    if (P > cap) { free(cs); free(zc); return -P; }
    opair *pr = (opair *)malloc(sizeof(opair) * (P > 0 ? P : 1));
    long n = 0;
    for (long c = 0; c < C; ++c) {
        const ocam *cm = cs + view_of(c, k, V, view_start);
        for (int ty = rect[4 * c + 1]; ty < rect[4 * c + 3]; ++ty)
            for (int tx = rect[4 * c]; tx < rect[4 * c + 2]; ++tx) {
                uint64_t tile = (uint64_t)(cm->tile_base + (long)ty * cm->TX + tx);
                pr[n].key = (tile << 32) | depth_bits[c];
                pr[n].val = (uint32_t)c;
                ++n;
            }
    }
    qsort(pr, P, sizeof(opair), pair_cmp);
    for (long i = 0; i < P; ++i) {
        keys[i] = pr[i].key;
        vals[i] = pr[i].val;
        uint32_t t = (uint32_t)(pr[i].key >> 32);
        if (i == 0 || (uint32_t)(pr[i - 1].key >> 32) != t) ranges[2 * t] = (uint32_t)i;
        if (i == P - 1 || (uint32_t)(pr[i + 1].key >> 32) != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
    free(pr); free(cs); free(zc);
    return P;
}

/* ------------------------------------------------------------------------ */
/* a4: Eq. 1 at one pixel over an ordered splat list.  C = sum_i c_i a_i T_i,
 * T_{i+1} = T_i (1 - a_i), a_i = min(0.99, o_i exp(power_i)); splats with
 * power > 0 or a_i < 1/255 are skipped; compositing stops before the splat
 * whose T' would fall below 1e-4.  Output C + T_final * bg. */

typedef struct {
    const double *mean2d, *conic, *opacity, *colour;
} osplats;

typedef struct {
    double C[3], T;
    long last;     /* 1-based list position of the last composited splat (0: none) */
    long nev;      /* list entries examined */
    int flag;      /* a decision lies within the band of its threshold */
    uint64_t hash;
} opix;

static void composite_pixel(const osplats *s, const uint32_t *list, long n, double px, double py,
                            const double bg[3], double band, double bandT, opix *out)
{
    double C[3] = {0, 0, 0}, T = 1.0;
    long last = 0, nev = 0;
    int flag = 0;
    uint64_t h = 1469598103934665603ULL;
    for (long j = 0; j < n; ++j) {
        uint32_t id = list[j];
        ++nev;
        double dx = s->mean2d[2 * id] - px, dy = s->mean2d[2 * id + 1] - py;
        const double *cn = s->conic + 3 * id;
        double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
        double pmag = 0.5 * (fabs(cn[0]) * dx * dx + fabs(cn[2]) * dy * dy) + fabs(cn[1] * dx * dy);
        if (power > 0.0 || -power <= band * pmag) flag = 1;
        if (power > 0.0) { fnv(&h, (uint64_t)j * 4 + 1); continue; }
        double ag = s->opacity[id] * exp(power);
        flag |= near_rel(ag, O_ALPHA_MAX, band) | near_rel(ag, O_ALPHA_MIN, band);
        double alpha = ag < O_ALPHA_MAX ? ag : O_ALPHA_MAX;
        if (!(ag < O_ALPHA_MAX)) fnv(&h, (uint64_t)j * 4);
        if (alpha < O_ALPHA_MIN) { fnv(&h, (uint64_t)j * 4 + 2); continue; }
        double Tn = T * (1.0 - alpha);
        flag |= near_rel(Tn, O_T_MIN, bandT);
        if (Tn < O_T_MIN) { fnv(&h, (uint64_t)j * 4 + 3); break; }
        for (int ch = 0; ch < 3; ++ch) C[ch] += s->colour[3 * id + ch] * alpha * T;
        T = Tn;
        last = j + 1;
    }
    for (int ch = 0; ch < 3; ++ch) out->C[ch] = C[ch] + T * bg[ch];
    out->T = T; out->last = last; out->nev = nev; out->flag = flag; out->hash = h;
}

static int cmp_depth_id(const void *pa, const void *pb)
{
    const opair *a = (const opair *)pa, *b = (const opair *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->val < b->val ? -1 : (a->val > b->val);
}

/* Builds the ordered list of one pixel.
 * mode 0: binned (the tile's range of the sorted pairs);
 * mode 1: brute, every splat of the view whose tile rectangle covers the
 *         pixel's tile, ordered by (depth bits, id);
 * mode 2: brute, every valid splat of the view (no tile cutoff), same order. */
static long pixel_list(int mode, const ocam *cm, int v, int px, int py, long C, int k, int V,
                       const long *view_start, const uint32_t *depth_bits, const int *rect,
                       const int *status, const uint32_t *ranges, const uint32_t *vals,
                       opair *scratch, uint32_t *list)
{
    int tx = px / O_TILE, ty = py / O_TILE;
    if (mode == 0) {
        long t = cm->tile_base + (long)ty * cm->TX + tx;
        long s = ranges[2 * t], e = ranges[2 * t + 1];
        for (long i = s; i < e; ++i) list[i - s] = vals[i];
        return e - s;
    }
    long n = 0;
    long c0 = view_start[v] * k, c1 = view_start[v + 1] * k;
    (void)C; (void)V;
    for (long c = c0; c < c1; ++c) {
        if (!status[c]) continue;
        if (mode == 1 && !(tx >= rect[4 * c] && tx < rect[4 * c + 2] && ty >= rect[4 * c + 1] &&
                           ty < rect[4 * c + 3]))
            continue;
        scratch[n].key = depth_bits[c];
        scratch[n].val = (uint32_t)c;
        ++n;
    }
    qsort(scratch, n, sizeof(opair), cmp_depth_id);
    for (long i = 0; i < n; ++i) list[i] = scratch[i].val;
    return n;
}

int gso_render(int V, const int *wh, long C, int k, const long *view_start, const double *mean2d,
               const double *conic, const double *opacity, const double *colour,
               const uint32_t *depth_bits, const int *rect, const int *status, int mode,
               const uint32_t *ranges, const uint32_t *vals, const double *bg, double band,
               double bandT, double *image, double *T_final, int *last, long *nev,
               unsigned char *pix_flag, uint64_t *hash)
{
    ocam *cs = (ocam *)calloc(V, sizeof(ocam));
    double *zc = (double *)calloc(16 * (size_t)V, sizeof(double));
    load_cams(V, zc, wh, cs);
    osplats s = {mean2d, conic, opacity, colour};
    long maxn = C > 0 ? C : 1;
    opair *scratch = (opair *)malloc(sizeof(opair) * maxn);
    uint32_t *list = (uint32_t *)malloc(sizeof(uint32_t) * (mode == 0 ? (maxn * 64 + 1) : maxn));
    long list_cap = mode == 0 ? maxn * 64 + 1 : maxn;
    uint64_t H = 1469598103934665603ULL;
    long total_ev = 0;
    for (int v = 0; v < V; ++v) {
        const ocam *cm = cs + v;
        long W = cm->W, Hh = cm->H;
        double *img = image + 3 * cm->pix_base;
        for (int py = 0; py < Hh; ++py)
            for (int px = 0; px < W; ++px) {
                long n;
                if (mode == 0) {
                    long t = cm->tile_base + (long)(py / O_TILE) * cm->TX + px / O_TILE;
                    n = (long)ranges[2 * t + 1] - (long)ranges[2 * t];
                    if (n > list_cap) {
                        free(list);
                        list_cap = n;
                        list = (uint32_t *)malloc(sizeof(uint32_t) * list_cap);
                    }
                }
                n = pixel_list(mode, cm, v, px, py, C, k, V, view_start, depth_bits, rect,
                               status, ranges, vals, scratch, list);
                opix o;
                composite_pixel(&s, list, n, (double)px, (double)py, bg, band, bandT, &o);
                long pi = (long)py * W + px;
                for (int ch = 0; ch < 3; ++ch) img[(long)ch * W * Hh + pi] = o.C[ch];
                if (T_final) T_final[cm->pix_base + pi] = o.T;
                if (last) last[cm->pix_base + pi] = (int)o.last;
                if (pix_flag) pix_flag[cm->pix_base + pi] = (unsigned char)o.flag;
                total_ev += o.nev;
                fnv(&H, o.hash);
            }
    }
    if (nev) *nev = total_ev;
    if (hash) *hash = H;
    free(scratch); free(list); free(cs); free(zc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a5: L = sum over views of mean_{pixel,channel} |C - C_target| (L1 term of
 * Eq. 3); dL/dC = sign(C - C_target) / (3 H W). */
double gso_l1(int V, const int *wh, const double *image, const double *target, double *dimage)
{
    double L = 0;
    long base = 0;
    for (int v = 0; v < V; ++v) {
        long n = 3L * wh[2 * v] * wh[2 * v + 1];
        double s = 0;
        for (long i = 0; i < n; ++i) {
            double d = image[base + i] - target[base + i];
            s += fabs(d);
            if (dimage) dimage[base + i] = (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
        }
        L += s / (double)n;
        base += n;
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Structural term of Eq. 3.  The paper takes its objective from the 3DGS
 * work it cites: L = lambda L1 + (1 - lambda) L_SSIM with L_SSIM = 1 - SSIM.
 * Readings (the paper gives no constants): SSIM of one view is the mean over
 * pixels and channels of the SSIM map computed per channel with an 11x11
 * Gaussian window (sigma 1.5, normalised to sum 1), zero padding outside the
 * image ("same" size), C1 = 0.01^2, C2 = 0.03^2; L_SSIM is summed over the
 * views like the L1 term.  For pixel p of one channel, with window weights
 * G(i, j) and x, y the rendered and target images:
 *   mu_x = sum G x,  mu_y = sum G y,  s_xx = sum G x^2,  s_yy = sum G y^2,
 *   s_xy = sum G x y (sums over the window, zero outside the image),
 *   var_x = s_xx - mu_x^2,  var_y = s_yy - mu_y^2,  cov = s_xy - mu_x mu_y,
 *   S = (2 mu_x mu_y + C1)(2 cov + C2) / ((mu_x^2 + mu_y^2 + C1)(var_x + var_y + C2)).
 * Reverse (derived by hand): with A1 = 2 mu_x mu_y + C1, A2 = 2 cov + C2,
 * B1 = mu_x^2 + mu_y^2 + C1, B2 = var_x + var_y + C2,
 *   dS/dmu_x = 2 mu_y A2 / (B1 B2) - 2 mu_x S / B1 + 2 mu_x S / B2 - 2 mu_y A1 / (B1 B2)
 *   dS/ds_xx = -S / B2,   dS/ds_xy = 2 A1 / (B1 B2),
 * and d/dx(r) = sum over the pixels p whose window holds r of
 *   G(r - p) (dS/dmu_x(p) + 2 x(r) dS/ds_xx(p) + y(r) dS/ds_xy(p)).
 * Returns L_SSIM = sum over views of (1 - mean S); ssim_map (3HW per view,
 * nullable) receives S, dimage (nullable) dL_SSIM/dimage. */
#define O_SSIM_R 5
static void ssim_window(double g[2 * O_SSIM_R + 1])
{
    double sum = 0;
    for (int i = -O_SSIM_R; i <= O_SSIM_R; ++i) {
        g[i + O_SSIM_R] = exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
        sum += g[i + O_SSIM_R];
    }
    for (int i = 0; i < 2 * O_SSIM_R + 1; ++i) g[i] /= sum;
}

double gso_ssim(int V, const int *wh, const double *image, const double *target, double *ssim_map,
                double *dimage)
{
    const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
    double g[2 * O_SSIM_R + 1];
    ssim_window(g);
    double L = 0;
    long base = 0;
    for (int v = 0; v < V; ++v) {
        const int W = wh[2 * v], H = wh[2 * v + 1];
        const long np = (long)W * H, n = 3 * np;
        double *dmu = malloc(sizeof(double) * np), *dsxx = malloc(sizeof(double) * np);
        double *dsxy = malloc(sizeof(double) * np);
        double ssum = 0;
        for (int ch = 0; ch < 3; ++ch) {
            const double *x = image + base + ch * np, *y = target + base + ch * np;
            for (int py = 0; py < H; ++py)
                for (int px = 0; px < W; ++px) {
                    double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
                    for (int j = -O_SSIM_R; j <= O_SSIM_R; ++j)
                        for (int i = -O_SSIM_R; i <= O_SSIM_R; ++i) {
                            const int qx = px + i, qy = py + j;
                            if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                            const double w = g[i + O_SSIM_R] * g[j + O_SSIM_R];
                            const double a = x[(long)qy * W + qx], b = y[(long)qy * W + qx];
                            mx += w * a; my += w * b;
                            sxx += w * a * a; syy += w * b * b; sxy += w * a * b;
                        }
                    const double vx = sxx - mx * mx, vy = syy - my * my, cv = sxy - mx * my;
                    const double A1 = 2 * mx * my + C1, A2 = 2 * cv + C2;
                    const double B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
                    const double S = A1 * A2 / (B1 * B2);
                    const long p = (long)py * W + px;
                    if (ssim_map) ssim_map[base + ch * np + p] = S;
                    ssum += S;
                    dmu[p] = 2 * my * A2 / (B1 * B2) - 2 * mx * S / B1 + 2 * mx * S / B2 - 2 * my * A1 / (B1 * B2);
                    dsxx[p] = -S / B2;
                    dsxy[p] = 2 * A1 / (B1 * B2);
                }
            if (dimage) {
                /* d(1 - mean S)/dS = -1 / n */
                for (int ry = 0; ry < H; ++ry)
                    for (int rx = 0; rx < W; ++rx) {
                        const long r = (long)ry * W + rx;
                        double acc = 0;
                        for (int j = -O_SSIM_R; j <= O_SSIM_R; ++j)
                            for (int i = -O_SSIM_R; i <= O_SSIM_R; ++i) {
                                const int qx = rx - i, qy = ry - j;   /* p = r - (i, j): r = p + (i, j) */
                                if (qx < 0 || qx >= W || qy < 0 || qy >= H) continue;
                                const double w = g[i + O_SSIM_R] * g[j + O_SSIM_R];
                                const long q = (long)qy * W + qx;
                                acc += w * (dmu[q] + 2 * x[r] * dsxx[q] + y[r] * dsxy[q]);
                            }
                        dimage[base + ch * np + r] = -acc / (double)n;
                    }
            }
        }
        L += 1.0 - ssum / (double)n;
        free(dmu); free(dsxx); free(dsxy);
        base += n;
    }
    return L;
}

/* ------------------------------------------------------------------------ */
/* Optimizer step.  The paper minimises Eq. 3 by gradient-based refinement of
 * the anchor features, offsets, scalings and decoder weights (Sec. III,
 * "System Overview"; the anchor positions themselves change only at loop
 * closures); the optimizer is the one of the 3DGS / Scaffold-GS training the
 * paper builds on: Adam with bias correction.  In place, one tensor:
 *   m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *   p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
void gso_adam(long n, double *param, const double *grad, double *m, double *v, long step, double lr, double b1,
              double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        param[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* Densification statistics of the incremental Scaffold-GS growth and pruning
 * the paper adopts (Sec. III, "System Overview": refinement, densification
 * and pruning).  Accumulated over the rows (view, anchor) of one iteration:
 *   every row:  anchor_denom[a] += 1,
 *               opacity_accum[a] += sum over its k Gaussians of max(opacity, 0);
 *   every rendered Gaussian (row, i) (tiles > 0):
 *               grad_accum[a k + i] += |dL/d mean2d| (pixel units),
 *               offset_denom[a k + i] += 1.
 * sgrad: 9 floats per candidate, the first two dL/d mean2d. */
void gso_densify_stats(long rows, int k, const int *row_anchor, const int *tiles, const double *opacity,
                       const double *sgrad, double *grad_accum, int *offset_denom, double *opacity_accum,
                       int *anchor_denom)
{
    for (long r = 0; r < rows; ++r) {
        const int a = row_anchor[r];
        double so = 0;
        for (int i = 0; i < k; ++i) {
            const long c = r * k + i;
            so += opacity[c] > 0 ? opacity[c] : 0.0;
            if (tiles[c] > 0) {
                const double gx = sgrad[9 * c], gy = sgrad[9 * c + 1];
                grad_accum[(long)a * k + i] += sqrt(gx * gx + gy * gy);
                offset_denom[(long)a * k + i] += 1;
            }
        }
        opacity_accum[a] += so;
        anchor_denom[a] += 1;
    }
}

/* Growth / pruning candidates from the statistics, with the caller's
 * thresholds (the paper states none): an offset grows where it was rendered
 * in at least min_count views and its mean gradient norm is >= grad_thr; an
 * anchor is pruned where it was visible in at least min_count views and its
 * mean opacity sum is < opacity_thr.  The means are taken in single precision
 * (float accumulators divided by their counts), as the device computes them. */
void gso_densify_masks(long N, int k, const float *grad_accum, const int *offset_denom, const float *opacity_accum,
                       const int *anchor_denom, float grad_thr, float opacity_thr, int min_count,
                       unsigned char *grow, unsigned char *prune)
{
    for (long j = 0; j < N * k; ++j) {
        const int d = offset_denom[j];
        grow[j] = (unsigned char)(d >= min_count && d > 0 && grad_accum[j] / (float)d >= grad_thr);
    }
    for (long a = 0; a < N; ++a) {
        const int d = anchor_denom[a];
        prune[a] = (unsigned char)(d >= min_count && d > 0 && opacity_accum[a] / (float)d < opacity_thr);
    }
}

/* ------------------------------------------------------------------------ */
/* Map maintenance.
 *
 * Voxelisation, Eq. 4: V = unique(round(P / eps)) * eps.  Reading: round to
 * the nearest integer with ties to even, the quotient and the rounding taken
 * in single precision (p / eps as one correctly rounded float division, the
 * precision the device decides in); voxel index (i, j, l) is packed into the
 * 64-bit key ((i + 2^20) << 42) | ((j + 2^20) << 21) | (l + 2^20), so indices
 * must satisfy |index| < 2^20.  The output is the keys in ascending order that
 * are not in `existing` (sorted ascending; the anchors already in the map),
 * with their centres index * eps (one float multiply).  Returns the count,
 * -(count) when it exceeds cap (nothing past cap written), or LONG_MIN when an
 * index is out of range. */
static int cmp_u64(const void *a, const void *b)
{
    const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

long gso_voxelize(long P, const float *pts, float eps, const uint64_t *existing, long n_existing, uint64_t *keys_out,
                  float *centers_out, long cap)
{
    const float lim = 1048576.0f;   /* 2^20 */
    uint64_t *k = (uint64_t *)malloc(sizeof(uint64_t) * (P > 0 ? P : 1));
    for (long i = 0; i < P; ++i) {
        uint64_t key = 0;
        for (int a = 0; a < 3; ++a) {
            const float q = pts[3 * i + a] / eps;
            const float r = rintf(q);
            if (!(r > -lim && r < lim)) { free(k); return LONG_MIN; }
            key = (key << 21) | (uint64_t)((long)r + 1048576L);
        }
        k[i] = key;
    }
    qsort(k, (size_t)P, sizeof(uint64_t), cmp_u64);
    long n = 0;
    for (long i = 0; i < P; ++i) {
        if (i > 0 && k[i] == k[i - 1]) continue;
        if (n_existing > 0 && bsearch(&k[i], existing, (size_t)n_existing, sizeof(uint64_t), cmp_u64)) continue;
        if (n < cap) {
            keys_out[n] = k[i];
            for (int a = 0; a < 3; ++a) {
                const long idx = (long)((k[i] >> (42 - 21 * a)) & 0x1FFFFF) - 1048576L;
                centers_out[3 * n + a] = (float)idx * eps;
            }
        }
        ++n;
    }
    free(k);
    return n <= cap ? n : -n;
}

/* Loop-closure deformation, Eq. 7.  For keyframe i with old and new
 * world-to-camera poses T_old,i and T_new,i, Delta T_i = T_new,i^-1 T_old,i
 * maps an anchor x to R_new^T (R_old x + t_old - t_new).  It applies to the
 * anchors inside keyframe i's local view frustum; readings: that frustum is
 * the visibility rule of the decoder (in front of the near plane 0.2, inside
 * the image grown by 15 % per side, under the old pose) cut at depth z_far,
 * and an anchor inside several corrected frusta takes the transform of the
 * nearest keyframe (smallest distance to the old camera centre, lowest index
 * on ties).  Anchors outside every frustum keep their position.  assigned[a]
 * = the keyframe used, or -1; flag[a] marks decisions within `band`
 * (relative) of a frustum edge or of a tie, which single precision may take
 * differently. */
void gso_loop_closure(int N, const double *xyz, int K, const double *cams_old, const double *cams_new,
                      const int *wh, double z_far, double band, double *xyz_out, int *assigned, unsigned char *flag)
{
    ocam *co = (ocam *)malloc(sizeof(ocam) * (K > 0 ? K : 1));
    ocam *cn = (ocam *)malloc(sizeof(ocam) * (K > 0 ? K : 1));
    load_cams(K, cams_old, wh, co);
    load_cams(K, cams_new, wh, cn);
    for (int a = 0; a < N; ++a) {
        const double *x = xyz + 3 * a;
        int best = -1, fl = 0;
        double bd = 0, second = -1;
        for (int i = 0; i < K; ++i) {
            const ocam *c = co + i;
            double p[3];
            to_cam(c, x, p);
            fl |= near_rel(p[2], O_NEAR, band) || near_rel(p[2], z_far, band);
            if (!(p[2] > O_NEAR && p[2] <= z_far)) continue;
            const double lox = -O_MARGIN * c->W, hix = (1.0 + O_MARGIN) * c->W;
            const double loy = -O_MARGIN * c->H, hiy = (1.0 + O_MARGIN) * c->H;
            const double u = c->fx * p[0] / p[2] + c->cx, w = c->fy * p[1] / p[2] + c->cy;
            fl |= fabs(u - lox) <= band * (fabs(lox) + 1) || fabs(u - hix) <= band * hix ||
                  fabs(w - loy) <= band * (fabs(loy) + 1) || fabs(w - hiy) <= band * hiy;
            if (!(u >= lox && u < hix && w >= loy && w < hiy)) continue;
            const double d = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
            if (best < 0 || d < bd) {
                second = best < 0 ? -1 : bd;
                best = i;
                bd = d;
            } else if (second < 0 || d < second) {
                second = d;
            }
        }
        if (best >= 0 && second >= 0 && fabs(second - bd) <= band * bd) fl = 1;
        double y[3] = {x[0], x[1], x[2]};
        if (best >= 0) {
            const ocam *o = co + best, *n = cn + best;
            double p[3];
            to_cam(o, x, p);
            const double q[3] = {p[0] - n->t[0], p[1] - n->t[1], p[2] - n->t[2]};
            for (int r = 0; r < 3; ++r) y[r] = n->R[r] * q[0] + n->R[3 + r] * q[1] + n->R[6 + r] * q[2];
        }
        xyz_out[3 * a] = y[0]; xyz_out[3 * a + 1] = y[1]; xyz_out[3 * a + 2] = y[2];
        assigned[a] = best;
        if (flag) flag[a] = (unsigned char)fl;
    }
    free(co); free(cn);
}

/* ------------------------------------------------------------------------ */
/* a6 (first half): reverse pass of Eq. 1 at one pixel.  With the composited
 * splats i (in order), weights w_i = a_i T_i and the colour carried by
 * everything behind splat i, B_i = sum_{j>i} c_j w_j + T_final bg:
 *   dL/dc_i     = w_i g
 *   dL/da_i     = g . (c_i T_i - B_i / (1 - a_i))
 *   a_i = o_i G_i (unclamped) => dL/do_i = dL/da_i G_i, dL/dpower_i = dL/da_i a_i
 *   clamped (o_i G_i >= 0.99) => no gradient to o_i or the Gaussian.
 * power = -(ca dx^2 + cc dy^2)/2 - cb dx dy with (dx,dy) = mean2d - pixel. */
int gso_render_bwd(int V, const int *wh, long C, const double *mean2d, const double *conic,
                   const double *opacity, const double *colour, const uint32_t *ranges,
                   const uint32_t *vals, const double *bg, const double *dimage,
                   double *dmean2d, double *dconic, double *dopacity, double *dcolour)
{
    ocam *cs = (ocam *)calloc(V, sizeof(ocam));
    double *zc = (double *)calloc(16 * (size_t)V, sizeof(double));
    load_cams(V, zc, wh, cs);
    for (long c = 0; c < C; ++c) {
        dmean2d[2 * c] = dmean2d[2 * c + 1] = 0;
        dconic[3 * c] = dconic[3 * c + 1] = dconic[3 * c + 2] = 0;
        dopacity[c] = 0;
        dcolour[3 * c] = dcolour[3 * c + 1] = dcolour[3 * c + 2] = 0;
    }
    long maxlist = 1;
    for (int v = 0; v < V; ++v)
        for (long t = cs[v].tile_base; t < cs[v].tile_base + (long)cs[v].TX * cs[v].TY; ++t) {
            long n = (long)ranges[2 * t + 1] - ranges[2 * t];
            if (n > maxlist) maxlist = n;
        }
    uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * maxlist);
    double *al = (double *)malloc(sizeof(double) * maxlist);
    double *Ti = (double *)malloc(sizeof(double) * maxlist);
    double *Gi = (double *)malloc(sizeof(double) * maxlist);
    int *clamped = (int *)malloc(sizeof(int) * maxlist);
    for (int v = 0; v < V; ++v) {
        const ocam *cm = cs + v;
        long W = cm->W, Hh = cm->H;
        const double *dimg = dimage + 3 * cm->pix_base;
        for (int py = 0; py < Hh; ++py)
            for (int px = 0; px < W; ++px) {
                long t = cm->tile_base + (long)(py / O_TILE) * cm->TX + px / O_TILE;
                long s0 = ranges[2 * t], e0 = ranges[2 * t + 1];
                /* forward again, recording the composited splats */
                double T = 1.0;
                long m = 0;
                for (long j = s0; j < e0; ++j) {
                    uint32_t id = vals[j];
                    double dx = mean2d[2 * id] - px, dy = mean2d[2 * id + 1] - py;
                    const double *cn = conic + 3 * id;
                    double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
                    if (power > 0.0) continue;
                    double G = exp(power);
                    double ag = opacity[id] * G;
                    double alpha = ag < O_ALPHA_MAX ? ag : O_ALPHA_MAX;
                    if (alpha < O_ALPHA_MIN) continue;
                    double Tn = T * (1.0 - alpha);
                    if (Tn < O_T_MIN) break;
                    ids[m] = id; al[m] = alpha; Ti[m] = T; Gi[m] = G;
                    clamped[m] = !(ag < O_ALPHA_MAX);
                    ++m;
                    T = Tn;
                }
                double g[3];
                long pi = (long)py * W + px;
                for (int ch = 0; ch < 3; ++ch) g[ch] = dimg[(long)ch * W * Hh + pi];
                /* B_i from the back: B_{m-1} = T_final bg, B_{i-1} = B_i + c_i w_i */
                double B[3] = {T * bg[0], T * bg[1], T * bg[2]};
                for (long i = m - 1; i >= 0; --i) {
                    uint32_t id = ids[i];
                    double w = al[i] * Ti[i];
                    double dal = 0;
                    for (int ch = 0; ch < 3; ++ch) {
                        dcolour[3 * id + ch] += w * g[ch];
                        dal += g[ch] * (colour[3 * id + ch] * Ti[i] - B[ch] / (1.0 - al[i]));
                    }
                    for (int ch = 0; ch < 3; ++ch) B[ch] += colour[3 * id + ch] * w;
                    if (clamped[i]) continue;
                    dopacity[id] += dal * Gi[i];
                    double dpow = dal * al[i];
                    double dx = mean2d[2 * id] - px, dy = mean2d[2 * id + 1] - py;
                    const double *cn = conic + 3 * id;
                    dmean2d[2 * id] += dpow * (-(cn[0] * dx + cn[1] * dy));
                    dmean2d[2 * id + 1] += dpow * (-(cn[2] * dy + cn[1] * dx));
                    dconic[3 * id] += dpow * (-0.5 * dx * dx);
                    dconic[3 * id + 1] += dpow * (-dx * dy);
                    dconic[3 * id + 2] += dpow * (-0.5 * dy * dy);
                }
            }
    }
    free(ids); free(al); free(Ti); free(Gi); free(clamped); free(cs); free(zc);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a6 (second half): chain rule of the projection, from per-splat gradients
 * (mean2d, conic, opacity, colour) to (mu, scale, quaternion, opacity,
 * colour) of the 3D Gaussian.  Culled splats get zero gradient. */
int gso_project_bwd(long C, int k, int V, const long *view_start, const double *cams,
                    const int *wh, const double *mu, const double *scale, const double *quat,
                    const int *status, const double *dmean2d, const double *dconic,
                    double *dmu, double *dscale, double *dquat)
{
    ocam *cs = (ocam *)malloc(sizeof(ocam) * V);
    load_cams(V, cams, wh, cs);
    for (long c = 0; c < C; ++c) {
        for (int j = 0; j < 3; ++j) dmu[3 * c + j] = dscale[3 * c + j] = 0;
        for (int j = 0; j < 4; ++j) dquat[4 * c + j] = 0;
        if (!status[c]) continue;
        const ocam *cm = cs + view_of(c, k, V, view_start);
        const double *R = cm->R;
        double p[3];
        to_cam(cm, mu + 3 * c, p);
        double Rq[9], S3[9];
        const double *q = quat + 4 * c;
        quat_to_rot(q, Rq);
        const double *s = scale + 3 * c;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += Rq[3 * i + l] * s[l] * s[l] * Rq[3 * j + l];
                S3[3 * i + j] = acc;
            }
        double limx = O_TANCLAMP * (cm->W / (2.0 * cm->fx));
        double limy = O_TANCLAMP * (cm->H / (2.0 * cm->fy));
        double ux = p[0] / p[2], uy = p[1] / p[2];
        int inx = ux >= -limx && ux <= limx, iny = uy >= -limy && uy <= limy;
        double txz = inx ? ux : (ux < 0 ? -limx : limx);
        double tyz = iny ? uy : (uy < 0 ? -limy : limy);
        double fx = cm->fx, fy = cm->fy, z = p[2];
        double J[6] = {fx / z, 0.0, -fx * txz / z, 0.0, fy / z, -fy * tyz / z};
        double T[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[3 * i + j] = J[3 * i] * R[j] + J[3 * i + 1] * R[3 + j] + J[3 * i + 2] * R[6 + j];
        double S2[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l)
                    for (int m = 0; m < 3; ++m) acc += T[3 * i + l] * S3[3 * l + m] * T[3 * j + m];
                S2[2 * i + j] = acc;
            }
        double a = S2[0] + O_LOWPASS, b = S2[1], cc = S2[3] + O_LOWPASS;
        double det = a * cc - b * b, d2 = det * det;
        /* conic (ca, cb, cc') = (cc, -b, a)/det  ->  gradient on (a, b, cc) */
        const double *dk = dconic + 3 * c;
        double da = (dk[0] * (-cc * cc) + dk[1] * (b * cc) + dk[2] * (-b * b)) / d2;
        double db = (dk[0] * (2 * b * cc) + dk[1] * (-(a * cc + b * b)) + dk[2] * (2 * a * b)) / d2;
        double dc = (dk[0] * (-b * b) + dk[1] * (a * b) + dk[2] * (-a * a)) / d2;
        /* symmetric gradient of Sigma2 (b sits at (0,1) and (1,0)) */
        double G2[4] = {da, 0.5 * db, 0.5 * db, dc};
        /* Sigma2 = T S3 T^T: dS3 = T^T G2 T, dT = 2 G2 T S3 */
        double dS3[9], dT[6];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 2; ++l)
                    for (int m = 0; m < 2; ++m) acc += T[3 * l + i] * G2[2 * l + m] * T[3 * m + j];
                dS3[3 * i + j] = acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 2; ++l)
                    for (int m = 0; m < 3; ++m) acc += G2[2 * i + l] * T[3 * l + m] * S3[3 * m + j];
                dT[3 * i + j] = 2.0 * acc;
            }
        /* T = J R  ->  dJ = dT R^T */
        double dJ[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                dJ[3 * i + j] = dT[3 * i] * R[3 * j] + dT[3 * i + 1] * R[3 * j + 1] +
                                dT[3 * i + 2] * R[3 * j + 2];
        /* J entries as functions of p = (x, y, z):
         * J00 = fx/z, J02 = -fx clamp(x/z)/z, J11 = fy/z, J12 = -fy clamp(y/z)/z */
        double dp[3] = {0, 0, 0};
        dp[2] += dJ[0] * (-fx / (z * z)) + dJ[4] * (-fy / (z * z));
        /* J02 = -fx txz / z */
        dp[2] += dJ[2] * (fx * txz / (z * z));
        if (inx) { /* txz = x/z */
            dp[0] += dJ[2] * (-fx / (z * z));
            dp[2] += dJ[2] * (fx * p[0] / (z * z * z));
        }
        dp[2] += dJ[5] * (fy * tyz / (z * z));
        if (iny) {
            dp[1] += dJ[5] * (-fy / (z * z));
            dp[2] += dJ[5] * (fy * p[1] / (z * z * z));
        }
        /* mean2d = (fx x/z + cx, fy y/z + cy) */
        const double *dm = dmean2d + 2 * c;
        dp[0] += dm[0] * fx / z;
        dp[1] += dm[1] * fy / z;
        dp[2] += dm[0] * (-fx * p[0] / (z * z)) + dm[1] * (-fy * p[1] / (z * z));
        /* p = R mu + t  ->  dmu = R^T dp */
        for (int j = 0; j < 3; ++j) dmu[3 * c + j] = R[j] * dp[0] + R[3 + j] * dp[1] + R[6 + j] * dp[2];
        /* S3 = Mq Mq^T with Mq = Rq diag(s): dMq = 2 dS3 Mq */
        double Mq[9], dM[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Mq[3 * i + j] = Rq[3 * i + j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int l = 0; l < 3; ++l) acc += dS3[3 * i + l] * Mq[3 * l + j];
                dM[3 * i + j] = 2.0 * acc;
            }
        double dRq[9];
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int i = 0; i < 3; ++i) acc += dM[3 * i + j] * Rq[3 * i + j];
            dscale[3 * c + j] = acc;
            for (int i = 0; i < 3; ++i) dRq[3 * i + j] = dM[3 * i + j] * s[j];
        }
        /* rotation matrix of q = (w, x, y, z), differentiated entry by entry */
        double w = q[0], x = q[1], y = q[2], zq = q[3];
        double *dq = dquat + 4 * c;
        dq[0] = 2 * (-zq * dRq[1] + y * dRq[2] + zq * dRq[3] - x * dRq[5] - y * dRq[6] + x * dRq[7]);
        dq[1] = 2 * (y * dRq[1] + zq * dRq[2] + y * dRq[3] - 2 * x * dRq[4] - w * dRq[5] +
                     zq * dRq[6] + w * dRq[7] - 2 * x * dRq[8]);
        dq[2] = 2 * (-2 * y * dRq[0] + x * dRq[1] + w * dRq[2] + x * dRq[3] + zq * dRq[5] -
                     w * dRq[6] + zq * dRq[7] - 2 * y * dRq[8]);
        dq[3] = 2 * (-2 * zq * dRq[0] - w * dRq[1] + x * dRq[2] + w * dRq[3] - 2 * zq * dRq[4] +
                     y * dRq[5] + x * dRq[6] + y * dRq[7]);
    }
    free(cs);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* a7: reverse pass of the decoder (Eq. 6, Eq. 2), summed over views.
 * Per candidate: dz_opa = dopacity (1 - opacity^2); dz_col = dcolour c (1-c);
 * dz_scale = dscale exp(l) s (1 - s) with s the sigmoid, and dl[3:6] +=
 * dscale * scale; dz_q = (dq - q (q . dq)) / |z_q|; dx_a += dmu,
 * doffset = dmu exp(l[0:3]), dl[0:3] += dmu offset exp(l[0:3]).  Then each
 * head: db2 = dz, dW2 = dz hid^T, dpre = W2^T dz masked by pre > 0, db1 =
 * dpre, dW1 = dpre u^T, du = W1^T dpre; u = [f, d/|d|, |d|] gives df and,
 * through the direction and distance, dx_a.  Candidates that decoding culled
 * (opacity <= 0) carry zero gradient by construction. */
int gso_decode_bwd(int N, int F, int k, int Hd, int M, const double *xyz, const double *feat,
                   const double *log_scaling, const double *offsets, const int *part,
                   const double *mlp, int V, const double *cams, const int *wh, long rows,
                   const int *av_anchor, const long *view_start, const double *dmu,
                   const double *dscale, const double *dquat, const double *dopacity,
                   const double *dcolour, double *dxyz, double *dfeat, double *dlog_scaling,
                   double *doffsets, double *dmlp)
{
    ocam *cs = (ocam *)malloc(sizeof(ocam) * V);
    load_cams(V, cams, wh, cs);
    long msz = mlp_size(F, k, Hd);
    int din = F + 4;
    for (long i = 0; i < 3L * N; ++i) dxyz[i] = 0;
    for (long i = 0; i < (long)N * F; ++i) dfeat[i] = 0;
    for (long i = 0; i < 6L * N; ++i) dlog_scaling[i] = 0;
    for (long i = 0; i < 3L * N * k; ++i) doffsets[i] = 0;
    for (long i = 0; i < M * msz; ++i) dmlp[i] = 0;
    double *u = (double *)malloc(sizeof(double) * din);
    double *du = (double *)malloc(sizeof(double) * din);
    double *pre = (double *)malloc(sizeof(double) * 3 * Hd);
    double *hid = (double *)malloc(sizeof(double) * 3 * Hd);
    double *dpre = (double *)malloc(sizeof(double) * 3 * Hd);
    double *z = (double *)malloc(sizeof(double) * 3 * 7 * k);
    double *dz = (double *)malloc(sizeof(double) * 3 * 7 * k);
    (void)rows;
    for (int v = 0; v < V; ++v) {
        double xc[3];
        cam_centre(cs + v, xc);
        for (long r = view_start[v]; r < view_start[v + 1]; ++r) {
            int a = av_anchor[r];
            ohead h[3];
            head_ptrs(mlp + (long)part[a] * msz, F, k, Hd, h);
            double d[3], delta;
            make_input(xyz + 3 * a, feat + (long)a * F, F, xc, u, d, &delta);
            mlp_forward(h, Hd, u, pre, hid, z, 7 * k);
            const double *ls = log_scaling + 6 * a;
            for (int i = 0; i < 3 * 7 * k; ++i) dz[i] = 0;
            for (int i = 0; i < k; ++i) {
                long c = r * k + i;
                double op = tanh(z[i]);
                if (!(op > 0.0)) continue;   /* culled by decoding: not rendered */
                dz[i] = dopacity[c] * (1.0 - op * op);
                for (int ch = 0; ch < 3; ++ch) {
                    double sc = sigm(z[7 * k + 3 * i + ch]);
                    dz[7 * k + 3 * i + ch] = dcolour[3 * c + ch] * sc * (1.0 - sc);
                }
                for (int j = 0; j < 3; ++j) {
                    double sg = sigm(z[14 * k + 7 * i + j]);
                    double e = exp(ls[3 + j]);
                    dz[14 * k + 7 * i + j] = dscale[3 * c + j] * e * sg * (1.0 - sg);
                    dlog_scaling[6 * a + 3 + j] += dscale[3 * c + j] * e * sg;
                }
                const double *qz = z + 14 * k + 7 * i + 3;
                double qn = sqrt(qz[0] * qz[0] + qz[1] * qz[1] + qz[2] * qz[2] + qz[3] * qz[3]);
                double qd = 0;
                for (int j = 0; j < 4; ++j) qd += (qz[j] / qn) * dquat[4 * c + j];
                for (int j = 0; j < 4; ++j)
                    dz[14 * k + 7 * i + 3 + j] = (dquat[4 * c + j] - (qz[j] / qn) * qd) / qn;
                const double *off = offsets + ((long)a * k + i) * 3;
                for (int j = 0; j < 3; ++j) {
                    double e = exp(ls[j]);
                    dxyz[3 * a + j] += dmu[3 * c + j];
                    doffsets[((long)a * k + i) * 3 + j] += dmu[3 * c + j] * e;
                    dlog_scaling[6 * a + j] += dmu[3 * c + j] * off[j] * e;
                }
            }
            for (int i = 0; i < din; ++i) du[i] = 0;
            double *dm = dmlp + (long)part[a] * msz;
            long hoff = 0;
            for (int hh = 0; hh < 3; ++hh) {
                int dout = h[hh].dout;
                double *dW1 = dm + hoff, *db1 = dW1 + (long)Hd * din;
                double *dW2 = db1 + Hd, *db2 = dW2 + (long)dout * Hd;
                hoff += (long)Hd * din + Hd + (long)dout * Hd + dout;
                const double *dzh = dz + hh * 7 * k;
                for (int o = 0; o < dout; ++o) {
                    db2[o] += dzh[o];
                    for (int j = 0; j < Hd; ++j) dW2[(long)o * Hd + j] += dzh[o] * hid[hh * Hd + j];
                }
                for (int j = 0; j < Hd; ++j) {
                    double s = 0;
                    for (int o = 0; o < dout; ++o) s += h[hh].W2[(long)o * Hd + j] * dzh[o];
                    dpre[hh * Hd + j] = pre[hh * Hd + j] > 0.0 ? s : 0.0;
                }
                for (int j = 0; j < Hd; ++j) {
                    db1[j] += dpre[hh * Hd + j];
                    for (int i = 0; i < din; ++i) {
                        dW1[(long)j * din + i] += dpre[hh * Hd + j] * u[i];
                        du[i] += h[hh].W1[(long)j * din + i] * dpre[hh * Hd + j];
                    }
                }
            }
            for (int i = 0; i < F; ++i) dfeat[(long)a * F + i] += du[i];
            /* u[F:F+3] = d / |d|, u[F+3] = |d|, d = x_a - x_c */
            double dir[3] = {d[0] / delta, d[1] / delta, d[2] / delta};
            double dd_dot = du[F] * dir[0] + du[F + 1] * dir[1] + du[F + 2] * dir[2];
            for (int j = 0; j < 3; ++j)
                dxyz[3 * a + j] += (du[F + j] - dir[j] * dd_dot) / delta + du[F + 3] * dir[j];
        }
    }
    free(u); free(du); free(pre); free(hid); free(dpre); free(z); free(dz); free(cs);
    return 0;
}

/* number of floats in one partition's packed MLP set */
long gso_mlp_size(int F, int k, int Hd) { return mlp_size(F, k, Hd); }
