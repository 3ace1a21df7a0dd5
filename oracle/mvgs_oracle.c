/*
 * mvgs_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, double-precision CPU reference for multi-view EWA splatting
 * (forward and backward).  It is the oracle the CUDA path is checked against;
 * nothing in the product library links, loads or calls it.  It shares no code,
 * header or constant table with the CUDA sources.
 *
 * What it computes, step by step (paper: Choi, Kim & Kim, "Efficient
 * multi-view training for 3D Gaussian Splatting", ICCV 2025):
 *   - Gaussian parameterisation mu, S, R, c, o and Sigma = R S S^T R^T (Sec. 3).
 *   - Projection of mu and Sigma to the image plane by the EWA local affine
 *     approximation Sigma' = J W Sigma W^T J^T (Sec. 3, citing Zwicker et al.).
 *   - Preprocessing: frustum culling, projection, duplication per covered tile,
 *     depth sort per tile (supplement, "Rasterization in multi-view training").
 *     The multi-view key holds tile, viewpoint and a 32-bit depth; here the
 *     (view, tile) pair is folded into one global tile id so the sort
 *     separates both.
 *   - Front-to-back alpha blending, Eq. 1: C(p) = sum_i c_i T_i o_i G_i(p).
 *   - Reverse-mode derivative of all of the above, summed over views
 *     (a Gaussian seen in several views gets gradients from each, Sec. 5.2).
 *
 * Constants the paper leaves to the 3DGS rasterizer it builds on (the paper
 * does not print them): low-pass dilation 0.3 px^2, alpha clamp 0.99, alpha
 * skip below 1/255, transmittance cutoff 1e-4, near plane from the camera,
 * 1.3x guard band on the Jacobian, 3-sigma radius with an eigenvalue floor of
 * 0.1, and a pixel support rule |p - mu'| <= r per axis so the image does not
 * depend on the tile size.
 *
 * Besides values it reports AMBIGUITY flags: decisions taken by comparing a
 * floating-point quantity with a threshold that lies within a small margin of
 * that threshold.  A float32 implementation may legitimately take the other
 * branch there, so tests compare such outputs loosely or not at all.
 *
 * Depth order is not such a decision: the sort key holds the float32 depth,
 * defined as the correctly rounded float32 of the camera-space depth, and an
 * implementation must produce exactly those bits; equal keys are ordered by
 * Gaussian index.
 *
 * Every array is dense over (view, Gaussian): record r = v * N + g.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- constants (3DGS conventions, see header comment) ------------------ */
static const double K_DILATION = 0.3;
static const double K_ALPHA_MAX = 0.99;
static const double K_ALPHA_MIN = 1.0 / 255.0;
static const double K_T_MIN = 1e-4;
static const double K_GUARD = 1.3;
static const double K_SIGMAS = 3.0;
static const double K_EIG_FLOOR = 0.1;

/* ---- ambiguity margins ------------------------------------------------- *
 * A decision is ambiguous when the compared quantity lies within the margin
 * of its threshold (a float32 evaluation may take the other branch) AND the
 * other branch would move the pixel by a non-negligible amount (M_EFFECT). */
static const double M_SUPPORT_PX = 2e-3;  /* |dx| vs r, pixels                  */
static const double M_ALPHA_REL = 2e-4;   /* alpha vs 1/255 and vs 0.99          */
static const double M_T_REL = 1e-3;       /* T(1-alpha) vs 1e-4                  */
static const double M_RADIUS_REL = 1e-4;  /* 3 sqrt(lambda) vs an integer        */
static const double M_CLAMP_ABS = 1e-5;   /* rgb vs 0, guard band                */
static const double M_EFFECT = 5e-6;      /* weight T alpha the flip would move  */

/* record-level ambiguity bits */
enum { RA_RADIUS = 1, RA_RGB_CLAMP = 2, RA_J_CLAMP = 4, RA_NEAR = 8 };
/* pixel-level ambiguity bits */
enum { PA_SUPPORT = 1, PA_ALPHA_MIN = 2, PA_T_MIN = 4, PA_ALPHA_MAX = 16, PA_RADIUS = 32 };

/* Camera record, passed as CAM_STRIDE doubles per view:
 * [0] width [1] height [2] fx [3] fy [4] cx [5] cy [6..14] R (world->camera,
 * row-major) [15..17] t [18..20] camera centre [21] near plane. */
#define CAM_STRIDE 22
typedef struct {
    int W, H;
    double fx, fy, cx, cy;
    double R[9], t[3], pos[3], near_z;
} cam_t;

static cam_t load_cam(const double* c) {
    cam_t k;
    k.W = (int)c[0];
    k.H = (int)c[1];
    k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
    for (int i = 0; i < 9; i++) k.R[i] = c[6 + i];
    for (int i = 0; i < 3; i++) { k.t[i] = c[15 + i]; k.pos[i] = c[18 + i]; }
    k.near_z = c[21];
    return k;
}

static int ceil_div(int a, int b) { return (a + b - 1) / b; }

/* ---- real spherical harmonics, degree <= 3 ------------------------------
 * Real SH basis with the Condon-Shortley phase kept, i.e. (-1)^m times the
 * usual real harmonics, ordered k = l^2 + l + m.  Normalisations are the
 * closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0)
 * written out per term. */
typedef struct { double c0, c1, c2a, c2b, c2c, c3a, c3b, c3c, c3d, c3e; } shk_t;

static shk_t sh_constants(void) {
    const double pi = 3.14159265358979323846;
    shk_t k;
    k.c0 = 0.5 * sqrt(1.0 / pi);
    k.c1 = sqrt(3.0 / (4.0 * pi));
    k.c2a = 0.5 * sqrt(15.0 / pi);
    k.c2b = 0.25 * sqrt(5.0 / pi);
    k.c2c = 0.25 * sqrt(15.0 / pi);
    k.c3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    k.c3b = 0.5 * sqrt(105.0 / pi);
    k.c3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    k.c3d = 0.25 * sqrt(7.0 / pi);
    k.c3e = 0.25 * sqrt(105.0 / pi);
    return k;
}

/* basis values Y[k] at unit direction (x, y, z); optionally dY[k][3] =
 * derivative of the basis polynomial with respect to (x, y, z). */
static void sh_eval(int deg, double x, double y, double z, double* Y, double (*dY)[3]) {
    shk_t k = sh_constants();
    int nk = (deg + 1) * (deg + 1);
    for (int i = 0; i < nk; i++) {
        Y[i] = 0.0;
        if (dY) dY[i][0] = dY[i][1] = dY[i][2] = 0.0;
    }
    Y[0] = k.c0;
    if (deg < 1) return;
    Y[1] = -k.c1 * y;
    Y[2] = k.c1 * z;
    Y[3] = -k.c1 * x;
    if (dY) {
        dY[1][1] = -k.c1;
        dY[2][2] = k.c1;
        dY[3][0] = -k.c1;
    }
    if (deg < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    Y[4] = k.c2a * x * y;
    Y[5] = -k.c2a * y * z;
    Y[6] = k.c2b * (2.0 * zz - xx - yy);
    Y[7] = -k.c2a * x * z;
    Y[8] = k.c2c * (xx - yy);
    if (dY) {
        dY[4][0] = k.c2a * y;        dY[4][1] = k.c2a * x;
        dY[5][1] = -k.c2a * z;       dY[5][2] = -k.c2a * y;
        dY[6][0] = -2.0 * k.c2b * x; dY[6][1] = -2.0 * k.c2b * y; dY[6][2] = 4.0 * k.c2b * z;
        dY[7][0] = -k.c2a * z;       dY[7][2] = -k.c2a * x;
        dY[8][0] = 2.0 * k.c2c * x;  dY[8][1] = -2.0 * k.c2c * y;
    }
    if (deg < 3) return;
    Y[9] = -k.c3a * y * (3.0 * xx - yy);
    Y[10] = k.c3b * x * y * z;
    Y[11] = -k.c3c * y * (4.0 * zz - xx - yy);
    Y[12] = k.c3d * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = -k.c3c * x * (4.0 * zz - xx - yy);
    Y[14] = k.c3e * z * (xx - yy);
    Y[15] = -k.c3a * x * (xx - 3.0 * yy);
    if (dY) {
        dY[9][0] = -6.0 * k.c3a * x * y;  dY[9][1] = -k.c3a * (3.0 * xx - 3.0 * yy);
        dY[10][0] = k.c3b * y * z;        dY[10][1] = k.c3b * x * z;   dY[10][2] = k.c3b * x * y;
        dY[11][0] = 2.0 * k.c3c * x * y;  dY[11][1] = -k.c3c * (4.0 * zz - xx - 3.0 * yy);
        dY[11][2] = -8.0 * k.c3c * y * z;
        dY[12][0] = -6.0 * k.c3d * x * z; dY[12][1] = -6.0 * k.c3d * y * z;
        dY[12][2] = k.c3d * (6.0 * zz - 3.0 * xx - 3.0 * yy);
        dY[13][0] = -k.c3c * (4.0 * zz - 3.0 * xx - yy); dY[13][1] = 2.0 * k.c3c * x * y;
        dY[13][2] = -8.0 * k.c3c * x * z;
        dY[14][0] = 2.0 * k.c3e * x * z;  dY[14][1] = -2.0 * k.c3e * y * z; dY[14][2] = k.c3e * (xx - yy);
        dY[15][0] = -k.c3a * (3.0 * xx - 3.0 * yy); dY[15][1] = 6.0 * k.c3a * x * y;
    }
}

void orc_sh_basis(int deg, int n, const double* dirs, double* out) {
    int nk = (deg + 1) * (deg + 1);
    for (int i = 0; i < n; i++) sh_eval(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], out + (size_t)i * nk, NULL);
}

/* ---- small linear algebra ----------------------------------------------- */
/* rotation matrix of the unit quaternion (w, x, y, z), row-major */
static void quat_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

void orc_quat_to_rotation(int n, const double* q, double* R) {
    for (int i = 0; i < n; i++) {
        double qq[4], nrm = 0.0;
        for (int j = 0; j < 4; j++) nrm += q[4 * i + j] * q[4 * i + j];
        nrm = sqrt(nrm);
        for (int j = 0; j < 4; j++) qq[j] = q[4 * i + j] / nrm;
        quat_rot(qq, R + 9 * i);
    }
}

/* Everything the forward derives for one Gaussian (view independent). */
typedef struct {
    double mu[3], s[3], qn[4], qnorm, R[9], M[9], Sig[9], o;
} gauss_t;

static gauss_t load_gauss(int g, const float* means, const float* log_scales, const float* quats, const float* logits) {
    gauss_t G;
    for (int i = 0; i < 3; i++) {
        G.mu[i] = means[3 * g + i];
        G.s[i] = exp((double)log_scales[3 * g + i]);
    }
    double n2 = 0.0;
    for (int i = 0; i < 4; i++) n2 += (double)quats[4 * g + i] * quats[4 * g + i];
    G.qnorm = sqrt(n2);
    for (int i = 0; i < 4; i++) G.qn[i] = quats[4 * g + i] / G.qnorm;
    quat_rot(G.qn, G.R);
    /* M = R diag(s); Sigma = M M^T */
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) G.M[3 * i + j] = G.R[3 * i + j] * G.s[j];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += G.M[3 * i + k] * G.M[3 * j + k];
            G.Sig[3 * i + j] = acc;
        }
    G.o = 1.0 / (1.0 + exp(-(double)logits[g]));
    return G;
}

/* View-dependent projection of one Gaussian. */
typedef struct {
    int visible;         /* passed the near test and has a non-empty rect   */
    double t[3];         /* camera-space mean                               */
    double tc[2];        /* guard-band clamped (tx, ty) used in J           */
    int clx, cly;        /* 0 = unclamped, +1 / -1 = clamped at +lim / -lim */
    double J[6];         /* 2x3, row-major                                  */
    double T[6];         /* J R_cam                                         */
    double a, b, c, det; /* Sigma' entries with the dilation                */
    double conic[3];     /* (A, B, C) = (c, -b, a) / det                    */
    double xy[2];
    double lam, r3;      /* largest eigenvalue and 3 sqrt(lam)              */
    int radius;
    int rect[4];         /* tile x0, y0, x1, y1 (exclusive ends)            */
    double dir[3], dlen; /* unit view direction from camera to mean         */
    double rgb_raw[3], rgb[3];
    int clampmask;
    int amb;
} proj_t;

static proj_t project_one(const gauss_t* G, const cam_t* cam, int deg, const float* sh_g, int tw, int th) {
    proj_t P;
    memset(&P, 0, sizeof(P));
    for (int i = 0; i < 3; i++)
        P.t[i] = cam->R[3 * i] * G->mu[0] + cam->R[3 * i + 1] * G->mu[1] + cam->R[3 * i + 2] * G->mu[2] + cam->t[i];
    double tz = P.t[2];
    if (fabs(tz - cam->near_z) < M_CLAMP_ABS) P.amb |= RA_NEAR;
    if (tz <= cam->near_z) return P;

    double limx = K_GUARD * 0.5 * cam->W / cam->fx;
    double limy = K_GUARD * 0.5 * cam->H / cam->fy;
    double ux = P.t[0] / tz, uy = P.t[1] / tz;
    if (fabs(fabs(ux) - limx) < M_CLAMP_ABS * limx) P.amb |= RA_J_CLAMP;
    if (fabs(fabs(uy) - limy) < M_CLAMP_ABS * limy) P.amb |= RA_J_CLAMP;
    P.clx = ux > limx ? 1 : (ux < -limx ? -1 : 0);
    P.cly = uy > limy ? 1 : (uy < -limy ? -1 : 0);
    P.tc[0] = (P.clx ? P.clx * limx : ux) * tz;
    P.tc[1] = (P.cly ? P.cly * limy : uy) * tz;

    P.J[0] = cam->fx / tz; P.J[1] = 0.0; P.J[2] = -cam->fx * P.tc[0] / (tz * tz);
    P.J[3] = 0.0; P.J[4] = cam->fy / tz; P.J[5] = -cam->fy * P.tc[1] / (tz * tz);
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += P.J[3 * i + k] * cam->R[3 * k + j];
            P.T[3 * i + j] = acc;
        }
    /* Sigma'_raw = T Sigma T^T */
    double TS[6];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += P.T[3 * i + k] * G->Sig[3 * k + j];
            TS[3 * i + j] = acc;
        }
    double cov[4];
    for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
            double acc = 0.0;
            for (int k = 0; k < 3; k++) acc += TS[3 * i + k] * P.T[3 * j + k];
            cov[2 * i + j] = acc;
        }
    P.a = cov[0] + K_DILATION;
    P.b = cov[1];
    P.c = cov[3] + K_DILATION;
    P.det = P.a * P.c - P.b * P.b;
    if (!(P.det > 0.0)) return P;
    P.conic[0] = P.c / P.det;
    P.conic[1] = -P.b / P.det;
    P.conic[2] = P.a / P.det;
    P.xy[0] = cam->fx * P.t[0] / tz + cam->cx;
    P.xy[1] = cam->fy * P.t[1] / tz + cam->cy;

    double mid = 0.5 * (P.a + P.c);
    double disc = mid * mid - P.det;
    P.lam = mid + sqrt(disc > K_EIG_FLOOR ? disc : K_EIG_FLOOR);
    P.r3 = K_SIGMAS * sqrt(P.lam);
    P.radius = (int)ceil(P.r3);
    {
        double fr = P.r3 - floor(P.r3);
        double m = M_RADIUS_REL * P.r3;
        if (fr < m || fr > 1.0 - m) P.amb |= RA_RADIUS;
    }
    int tiles_x = ceil_div(cam->W, tw), tiles_y = ceil_div(cam->H, th);
    /* Tiles the Gaussian covers: those that can hold a pixel centre where it
     * passes the support rule and alpha >= 1/255.  alpha >= 1/255 needs
     * d^T Sigma'^-1 d <= 2 ln(255 o); that ellipse's bounding box has
     * half-widths sqrt(2 ln(255 o) Sigma'_xx), sqrt(2 ln(255 o) Sigma'_yy).
     * The box is widened slightly (relative 1e-3 on the level, 1e-2 px) so
     * that it also covers every pixel a float32 evaluation lets through; the
     * image does not depend on the box, only the number of keys does. */
    double lvl = log(255.0 * G->o);
    if (!(lvl > 0.0)) return P;
    double ext = 2.0 * lvl * 1.001 + 1e-3;
    double r = (double)P.radius;
    double hx = sqrt(ext * P.a) + 1e-2, hy = sqrt(ext * P.c) + 1e-2;
    hx = hx < r ? hx : r;
    hy = hy < r ? hy : r;
    double fx0 = floor((P.xy[0] - hx) / tw), fx1 = floor((P.xy[0] + hx) / tw) + 1.0;
    double fy0 = floor((P.xy[1] - hy) / th), fy1 = floor((P.xy[1] + hy) / th) + 1.0;
    fx0 = fx0 < 0 ? 0 : (fx0 > tiles_x ? tiles_x : fx0);
    fx1 = fx1 < 0 ? 0 : (fx1 > tiles_x ? tiles_x : fx1);
    fy0 = fy0 < 0 ? 0 : (fy0 > tiles_y ? tiles_y : fy0);
    fy1 = fy1 < 0 ? 0 : (fy1 > tiles_y ? tiles_y : fy1);
    P.rect[0] = (int)fx0; P.rect[1] = (int)fy0; P.rect[2] = (int)fx1; P.rect[3] = (int)fy1;
    if (P.rect[0] >= P.rect[2] || P.rect[1] >= P.rect[3] || P.radius <= 0) return P;

    /* colour from SH at the direction camera -> mean */
    for (int i = 0; i < 3; i++) P.dir[i] = G->mu[i] - cam->pos[i];
    P.dlen = sqrt(P.dir[0] * P.dir[0] + P.dir[1] * P.dir[1] + P.dir[2] * P.dir[2]);
    for (int i = 0; i < 3; i++) P.dir[i] /= P.dlen;
    double Y[16];
    sh_eval(deg, P.dir[0], P.dir[1], P.dir[2], Y, NULL);
    int nk = (deg + 1) * (deg + 1);
    for (int ch = 0; ch < 3; ch++) {
        double acc = 0.0;
        for (int k = 0; k < nk; k++) acc += Y[k] * (double)sh_g[3 * k + ch];
        acc += 0.5;
        P.rgb_raw[ch] = acc;
        if (fabs(acc) < M_CLAMP_ABS) P.amb |= RA_RGB_CLAMP;
        if (acc < 0.0) { P.clampmask |= 1 << ch; acc = 0.0; }
        P.rgb[ch] = acc;
    }
    P.visible = 1;
    return P;
}

/* Dense projection of all (view, Gaussian) pairs.  Outputs are [V*N, ...]. */
void orc_project(int N, int deg, const float* means, const float* log_scales, const float* quats,
                 const float* logits, const float* sh, int V, const double* cams, int tw, int th,
                 int32_t* valid, double* xy, double* conic, double* cov, double* opac, double* rgb,
                 int32_t* clampmask, double* depth, int32_t* radius, int32_t* rect, int32_t* amb) {
    int nk = (deg + 1) * (deg + 1);
    for (int g = 0; g < N; g++) {
        gauss_t G = load_gauss(g, means, log_scales, quats, logits);
        for (int v = 0; v < V; v++) {
            cam_t cam = load_cam(cams + (size_t)v * CAM_STRIDE);
            proj_t P = project_one(&G, &cam, deg, sh + (size_t)g * nk * 3, tw, th);
            size_t r = (size_t)v * N + g;
            valid[r] = P.visible;
            xy[2 * r] = P.xy[0]; xy[2 * r + 1] = P.xy[1];
            for (int i = 0; i < 3; i++) {
                conic[3 * r + i] = P.conic[i];
                rgb[3 * r + i] = P.rgb[i];
            }
            cov[3 * r] = P.a; cov[3 * r + 1] = P.b; cov[3 * r + 2] = P.c;
            opac[r] = G.o;
            clampmask[r] = P.clampmask;
            depth[r] = P.t[2];
            radius[r] = P.visible ? P.radius : 0;
            for (int i = 0; i < 4; i++) rect[4 * r + i] = P.visible ? P.rect[i] : 0;
            amb[r] = P.amb;
        }
    }
}

/* ---- keys and sort ------------------------------------------------------ */
typedef struct { uint64_t key; int32_t g; int32_t rec; } entry_t;

static int cmp_entry(const void* pa, const void* pb) {
    const entry_t* a = (const entry_t*)pa;
    const entry_t* b = (const entry_t*)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->g != b->g) return a->g < b->g ? -1 : 1;
    return 0;
}

static uint32_t f32_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Number of (record, tile) keys; with a pixel window per view, only the
 * tiles that intersect the window are counted. */
int64_t orc_count_keys(int N, int V, int tw, int th, const int32_t* valid, const int32_t* rect,
                       const int32_t* window) {
    int64_t K = 0;
    for (int v = 0; v < V; v++)
        for (int g = 0; g < N; g++) {
            size_t r = (size_t)v * N + g;
            if (!valid[r]) continue;
            int x0 = rect[4 * r], y0 = rect[4 * r + 1], x1 = rect[4 * r + 2], y1 = rect[4 * r + 3];
            if (window) {
                int wx0 = window[4 * v] / tw, wx1 = (window[4 * v + 2] - 1) / tw + 1;
                int wy0 = window[4 * v + 1] / th, wy1 = (window[4 * v + 3] - 1) / th + 1;
                x0 = x0 > wx0 ? x0 : wx0; x1 = x1 < wx1 ? x1 : wx1;
                y0 = y0 > wy0 ? y0 : wy0; y1 = y1 < wy1 ? y1 : wy1;
                if (x1 <= x0 || y1 <= y0) continue;
            }
            K += (int64_t)(x1 - x0) * (y1 - y0);
        }
    return K;
}

/* Builds one key per (record, covered tile): high 32 bits = global tile id
 * (tiles of earlier views first), low 32 bits = float32 depth bits (depth > 0
 * so the bits order like the value); sorts by (key, Gaussian index) and
 * returns the sorted keys, sorted record ids (v*N+g) and per global tile the
 * range [start, end) into the sorted arrays.  `depth32` is the depth already
 * rounded to float32.  With a pixel window per view (x0, y0, x1, y1), only
 * keys of tiles that intersect the window are built. */
void orc_sort(int N, int V, const double* cams, int tw, int th, const int32_t* valid, const int32_t* rect,
              const float* depth32, const int32_t* window, int64_t K, uint64_t* keys_out, int32_t* recs_out,
              int64_t* ranges) {
    int64_t* tile_base = (int64_t*)malloc(sizeof(int64_t) * (V + 1));
    int* tiles_x = (int*)malloc(sizeof(int) * V);
    tile_base[0] = 0;
    for (int v = 0; v < V; v++) {
        cam_t cam = load_cam(cams + (size_t)v * CAM_STRIDE);
        tiles_x[v] = ceil_div(cam.W, tw);
        tile_base[v + 1] = tile_base[v] + (int64_t)tiles_x[v] * ceil_div(cam.H, th);
    }
    entry_t* E = (entry_t*)malloc(sizeof(entry_t) * (K > 0 ? K : 1));
    int64_t k = 0;
    for (int v = 0; v < V; v++)
        for (int g = 0; g < N; g++) {
            size_t r = (size_t)v * N + g;
            if (!valid[r]) continue;
            for (int ty = rect[4 * r + 1]; ty < rect[4 * r + 3]; ty++)
                for (int tx = rect[4 * r]; tx < rect[4 * r + 2]; tx++) {
                    if (window && (tx < window[4 * v] / tw || tx > (window[4 * v + 2] - 1) / tw ||
                                   ty < window[4 * v + 1] / th || ty > (window[4 * v + 3] - 1) / th))
                        continue;
                    uint64_t gt = (uint64_t)(tile_base[v] + (int64_t)ty * tiles_x[v] + tx);
                    E[k].key = (gt << 32) | f32_bits(depth32[r]);
                    E[k].g = g;
                    E[k].rec = (int32_t)r;
                    k++;
                }
        }
    qsort(E, (size_t)k, sizeof(entry_t), cmp_entry);
    int64_t T = tile_base[V];
    for (int64_t i = 0; i < 2 * T; i++) ranges[i] = 0;
    for (int64_t i = 0; i < k; i++) {
        keys_out[i] = E[i].key;
        recs_out[i] = E[i].rec;
        int64_t gt = (int64_t)(E[i].key >> 32);
        if (i == 0 || (int64_t)(E[i - 1].key >> 32) != gt) ranges[2 * gt] = i;
        if (i == k - 1 || (int64_t)(E[i + 1].key >> 32) != gt) ranges[2 * gt + 1] = i + 1;
    }
    free(E);
    free(tile_base);
    free(tiles_x);
}

/* ---- per-pixel blending (Eq. 1) ----------------------------------------- */
typedef struct {
    const double *xy, *conic, *opac, *rgb, *depth;
    const int32_t *radius, *amb;
} recs_t;

typedef struct {
    int32_t rec;
    double alpha, G, T; /* alpha, Gaussian falloff, transmittance before */
    double dx, dy;      /* pixel centre minus projected mean             */
    int clamped;        /* alpha hit the 0.99 clamp                      */
} contrib_t;

/* Walks one pixel's sorted list.  Fills the contributor list (if given) and
 * returns the number of contributors; writes colour, final T, the list
 * position one past the last contributor, ambiguity bits, (if given) a hash
 * of the contributor ids, so tests can tell when a perturbation changed a
 * discrete decision, and (if given) the expected depth sum alpha T z of the
 * contributors, the blend of Eq. 1 with each colour replaced by the camera
 * depth (the predicted depth the 3D D-SSIM of Sec. 5.1.2 lifts pixels with). */
static int blend_pixel(double px, double py, const int32_t* list, int64_t len, const recs_t* R, const double* bg,
                       double* C, double* Tout, int64_t* last, int* amb, contrib_t* out, int64_t cap,
                       uint64_t* hash, double* Dout) {
    double T = 1.0, D = 0.0;
    uint64_t h = 1469598103934665603ull;
    C[0] = C[1] = C[2] = 0.0;
    *last = 0;
    *amb = 0;
    int n = 0;
    for (int64_t i = 0; i < len; i++) {
        int32_t r = list[i];
        double mx = R->xy[2 * r], my = R->xy[2 * r + 1];
        double dx = px - mx, dy = py - my;
        double rad = (double)R->radius[r];
        double A = R->conic[3 * r], B = R->conic[3 * r + 1], Cc = R->conic[3 * r + 2];
        double power = -0.5 * (A * dx * dx + Cc * dy * dy) - B * dx * dy;
        double G = exp(power);
        double ag = R->opac[r] * G;
        double alpha = ag < K_ALPHA_MAX ? ag : K_ALPHA_MAX;
        double ex = fabs(dx) > fabs(dy) ? fabs(dx) : fabs(dy); /* Chebyshev distance to the mean */
        /* support rule; a record whose radius is ambiguous may cover one more pixel ring */
        int inside = fabs(dx) <= rad && fabs(dy) <= rad;
        if (alpha >= K_ALPHA_MIN * (1.0 - M_ALPHA_REL) && T * alpha >= M_EFFECT) {
            if (fabs(ex - rad) < M_SUPPORT_PX) *amb |= PA_SUPPORT;
            if ((R->amb[r] & RA_RADIUS) && ex > rad - 1.0 - M_SUPPORT_PX && ex <= rad + 1.0 + M_SUPPORT_PX)
                *amb |= PA_RADIUS;
        }
        if (!inside) continue;
        if (power > 0.0) continue;
        if (fabs(alpha - K_ALPHA_MIN) < M_ALPHA_REL * K_ALPHA_MIN && T * K_ALPHA_MIN >= M_EFFECT)
            *amb |= PA_ALPHA_MIN;
        if (alpha < K_ALPHA_MIN) continue;
        if (fabs(ag - K_ALPHA_MAX) < M_ALPHA_REL * K_ALPHA_MAX) *amb |= PA_ALPHA_MAX;
        double Tn = T * (1.0 - alpha);
        if (fabs(Tn - K_T_MIN) < M_T_REL * K_T_MIN && T * alpha >= M_EFFECT) *amb |= PA_T_MIN;
        if (Tn < K_T_MIN) break;
        for (int ch = 0; ch < 3; ch++) C[ch] += R->rgb[3 * r + ch] * alpha * T;
        D += R->depth[r] * alpha * T;
        if (out && n < cap) {
            out[n].rec = r;
            out[n].alpha = alpha;
            out[n].G = G;
            out[n].T = T;
            out[n].dx = dx;
            out[n].dy = dy;
            out[n].clamped = ag >= K_ALPHA_MAX;
        }
        n++;
        T = Tn;
        *last = i + 1;
        h = (h ^ (uint64_t)(uint32_t)r) * 1099511628211ull; /* FNV-1a over contributor ids */
    }
    for (int ch = 0; ch < 3; ch++) C[ch] += T * bg[ch];
    *Tout = T;
    if (hash) *hash = h;
    if (Dout) *Dout = D;
    return n;
}

typedef struct {
    int V;
    int64_t *tile_base, *pix_base;
    int *tiles_x;
    cam_t* cam;
} layout_t;

static layout_t make_layout(int V, const double* cams, int tw, int th) {
    layout_t L;
    L.V = V;
    L.tile_base = (int64_t*)malloc(sizeof(int64_t) * (V + 1));
    L.pix_base = (int64_t*)malloc(sizeof(int64_t) * (V + 1));
    L.tiles_x = (int*)malloc(sizeof(int) * V);
    L.cam = (cam_t*)malloc(sizeof(cam_t) * V);
    L.tile_base[0] = 0;
    L.pix_base[0] = 0;
    for (int v = 0; v < V; v++) {
        L.cam[v] = load_cam(cams + (size_t)v * CAM_STRIDE);
        L.tiles_x[v] = ceil_div(L.cam[v].W, tw);
        L.tile_base[v + 1] = L.tile_base[v] + (int64_t)L.tiles_x[v] * ceil_div(L.cam[v].H, th);
        L.pix_base[v + 1] = L.pix_base[v] + (int64_t)L.cam[v].W * L.cam[v].H;
    }
    return L;
}

static void free_layout(layout_t* L) {
    free(L->tile_base);
    free(L->pix_base);
    free(L->tiles_x);
    free(L->cam);
}

/* Renders all views (or a pixel window per view: window[4v..4v+3] = x0, y0,
 * x1, y1, exclusive ends; NULL = whole image).  Image layout: views
 * concatenated, each [3, H, W]; per-pixel arrays: views concatenated, [H, W].
 * Pixels outside the window are left untouched. */
void orc_render(int N, int V, const double* cams, int tw, int th, const double* bg, const double* xy,
                const double* conic, const double* opac, const double* rgb, const double* depth,
                const int32_t* radius, const int32_t* ramb, const int64_t* ranges, const int32_t* recs,
                const int32_t* window, double* img, double* Tfinal, int64_t* last, int32_t* pamb, uint64_t* chash,
                double* depth_out) {
    (void)N;
    layout_t L = make_layout(V, cams, tw, th);
    recs_t R = {xy, conic, opac, rgb, depth, radius, ramb};
    for (int v = 0; v < V; v++) {
        int W = L.cam[v].W, H = L.cam[v].H;
        int x0 = 0, y0 = 0, x1 = W, y1 = H;
        if (window) { x0 = window[4 * v]; y0 = window[4 * v + 1]; x1 = window[4 * v + 2]; y1 = window[4 * v + 3]; }
        for (int y = y0; y < y1; y++)
            for (int x = x0; x < x1; x++) {
                int64_t gt = L.tile_base[v] + (int64_t)(y / th) * L.tiles_x[v] + x / tw;
                int64_t s = ranges[2 * gt], e = ranges[2 * gt + 1];
                double C[3], T;
                int64_t lst;
                int a;
                uint64_t h;
                double D;
                blend_pixel(x + 0.5, y + 0.5, recs + s, e - s, &R, bg, C, &T, &lst, &a, NULL, 0, &h, &D);
                int64_t p = L.pix_base[v] + (int64_t)y * W + x;
                if (depth_out) depth_out[p] = D;
                if (chash) chash[p] = h;
                for (int ch = 0; ch < 3; ch++) img[3 * L.pix_base[v] + (int64_t)ch * W * H + (int64_t)y * W + x] = C[ch];
                Tfinal[p] = T;
                last[p] = lst;
                pamb[p] = a;
            }
    }
    free_layout(&L);
}

/* Per-pixel brute force without tiles: the records of view v that pass the
 * support rule at the pixel, ordered by (float32 depth, Gaussian index).
 * Used by tests to pin the tiled path; one pixel per call. */
typedef struct { uint32_t d; int32_t g; int32_t rec; } bf_t;
static int cmp_bf(const void* pa, const void* pb) {
    const bf_t* a = (const bf_t*)pa;
    const bf_t* b = (const bf_t*)pb;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    return a->g < b->g ? -1 : (a->g > b->g ? 1 : 0);
}

void orc_render_pixels_bruteforce(int N, int V, const double* cams, const double* bg, const int32_t* valid,
                                  const double* xy, const double* conic, const double* opac, const double* rgb,
                                  const double* depth, const int32_t* radius, const int32_t* ramb, int npix,
                                  const int32_t* pix /* [npix, 3] = v, x, y */, double* C_out, double* T_out,
                                  int32_t* ncontrib, int32_t* pamb) {
    (void)cams;
    recs_t R = {xy, conic, opac, rgb, depth, radius, ramb};
    bf_t* list = (bf_t*)malloc(sizeof(bf_t) * (N > 0 ? N : 1));
    int32_t* ids = (int32_t*)malloc(sizeof(int32_t) * (N > 0 ? N : 1));
    for (int i = 0; i < npix; i++) {
        int v = pix[3 * i], x = pix[3 * i + 1], y = pix[3 * i + 2];
        int n = 0;
        for (int g = 0; g < N; g++) {
            size_t r = (size_t)v * N + g;
            if (!valid[r]) continue;
            /* keep anything within radius + 1 so the support test (and its
             * ambiguity flag) is taken inside blend_pixel */
            double rad = radius[r] + 1.0 + 1e-3;
            if (fabs(x + 0.5 - xy[2 * r]) > rad || fabs(y + 0.5 - xy[2 * r + 1]) > rad) continue;
            list[n].d = f32_bits((float)depth[r]);
            list[n].g = g;
            list[n].rec = (int32_t)r;
            n++;
        }
        qsort(list, (size_t)n, sizeof(bf_t), cmp_bf);
        for (int k = 0; k < n; k++) ids[k] = list[k].rec;
        int64_t lst;
        int a;
        int nc = blend_pixel(x + 0.5, y + 0.5, ids, n, &R, bg, C_out + 3 * i, T_out + i, &lst, &a, NULL, 0, NULL, NULL);
        ncontrib[i] = nc;
        pamb[i] = a;
    }
    free(list);
    free(ids);
}

/* ---- backward of the blend ---------------------------------------------
 * Given dL/dimage (same layout as the image), accumulates per record r:
 *   g2d[9r + 0..1] dL/d mean2d (pixels)     g2d[9r + 2..4] dL/d conic (A, B, C)
 *   g2d[9r + 5]    dL/d opacity (activated) g2d[9r + 6..8] dL/d rgb
 *   e1[r]          sum over pixels of || dL/d mean2d contribution of that pixel ||
 * Derivatives of Eq. 1: dC/dc_i = alpha_i T_i and
 *   dC/dalpha_i = c_i T_i - (sum_{j>i} c_j alpha_j T_j + T_final bg) / (1 - alpha_i);
 * alpha = o G below the clamp (no derivative once clamped at 0.99);
 * G = exp(power), power = -(A dx^2 + C dy^2)/2 - B dx dy with d = p - mu'.
 * Pixels outside `window` (if given) are ignored. */
void orc_render_backward(int N, int V, const double* cams, int tw, int th, const double* bg, const double* xy,
                         const double* conic, const double* opac, const double* rgb, const double* depth,
                         const int32_t* radius, const int32_t* ramb, const int64_t* ranges, const int32_t* recs,
                         const int32_t* window, const double* dimg, double* g2d, double* e1) {
    layout_t L = make_layout(V, cams, tw, th);
    recs_t R = {xy, conic, opac, rgb, depth, radius, ramb};
    memset(g2d, 0, sizeof(double) * 9 * (size_t)N * V);
    memset(e1, 0, sizeof(double) * (size_t)N * V);
    int64_t maxlen = 1;
    for (int64_t t = 0; t < L.tile_base[V]; t++)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    contrib_t* cl = (contrib_t*)malloc(sizeof(contrib_t) * maxlen);
    for (int v = 0; v < V; v++) {
        int W = L.cam[v].W, H = L.cam[v].H;
        int x0 = 0, y0 = 0, x1 = W, y1 = H;
        if (window) { x0 = window[4 * v]; y0 = window[4 * v + 1]; x1 = window[4 * v + 2]; y1 = window[4 * v + 3]; }
        for (int y = y0; y < y1; y++)
            for (int x = x0; x < x1; x++) {
                int64_t gt = L.tile_base[v] + (int64_t)(y / th) * L.tiles_x[v] + x / tw;
                int64_t s = ranges[2 * gt], e = ranges[2 * gt + 1];
                double C[3], T;
                int64_t lst;
                int a;
                int n = blend_pixel(x + 0.5, y + 0.5, recs + s, e - s, &R, bg, C, &T, &lst, &a, cl, maxlen, NULL, NULL);
                double dC[3];
                for (int ch = 0; ch < 3; ch++)
                    dC[ch] = dimg[3 * L.pix_base[v] + (int64_t)ch * W * H + (int64_t)y * W + x];
                double S[3] = {T * bg[0], T * bg[1], T * bg[2]}; /* colour behind contributor i */
                for (int i = n - 1; i >= 0; i--) {
                    int32_t r = cl[i].rec;
                    double al = cl[i].alpha, Ti = cl[i].T;
                    double dLda = 0.0;
                    for (int ch = 0; ch < 3; ch++) {
                        double c = rgb[3 * r + ch];
                        g2d[9 * (size_t)r + 6 + ch] += dC[ch] * al * Ti;
                        dLda += dC[ch] * (c * Ti - S[ch] / (1.0 - al));
                    }
                    for (int ch = 0; ch < 3; ch++) S[ch] += rgb[3 * r + ch] * al * Ti;
                    if (cl[i].clamped) continue;
                    double G = cl[i].G, o = opac[r];
                    double dLdpow = dLda * o * G;
                    double dx = cl[i].dx, dy = cl[i].dy;
                    double A = conic[3 * r], B = conic[3 * r + 1], Cc = conic[3 * r + 2];
                    /* d power / d mu' = -(d power / d d) */
                    double gx = dLdpow * (A * dx + B * dy);
                    double gy = dLdpow * (Cc * dy + B * dx);
                    g2d[9 * (size_t)r + 0] += gx;
                    g2d[9 * (size_t)r + 1] += gy;
                    g2d[9 * (size_t)r + 2] += dLdpow * (-0.5 * dx * dx);
                    g2d[9 * (size_t)r + 3] += dLdpow * (-dx * dy);
                    g2d[9 * (size_t)r + 4] += dLdpow * (-0.5 * dy * dy);
                    g2d[9 * (size_t)r + 5] += dLda * G;
                    e1[r] += sqrt(gx * gx + gy * gy);
                }
            }
    }
    free(cl);
    free_layout(&L);
}

/* ---- backward of the projection ----------------------------------------
 * Chains the per-record 2D gradients (layout as in orc_render_backward) to
 * the Gaussian parameters and sums over views:
 *   g_means [N,3], g_log_scales [N,3], g_quats [N,4] (w,x,y,z, w.r.t. the raw
 *   quaternion before normalisation), g_logits [N], g_sh [N,(d+1)^2,3].
 * Outputs are overwritten. */
void orc_project_backward(int N, int deg, const float* means, const float* log_scales, const float* quats,
                          const float* logits, const float* sh, int V, const double* cams, int tw, int th,
                          const double* g2d, double* g_means, double* g_log_scales, double* g_quats,
                          double* g_logits, double* g_sh) {
    int nk = (deg + 1) * (deg + 1);
    for (int g = 0; g < N; g++) {
        gauss_t G = load_gauss(g, means, log_scales, quats, logits);
        const float* shg = sh + (size_t)g * nk * 3;
        double gmu[3] = {0, 0, 0}, gSig[9] = {0}, go = 0.0;
        double* gsh = g_sh + (size_t)g * nk * 3;
        for (int i = 0; i < nk * 3; i++) gsh[i] = 0.0;
        for (int v = 0; v < V; v++) {
            cam_t cam = load_cam(cams + (size_t)v * CAM_STRIDE);
            proj_t P = project_one(&G, &cam, deg, shg, tw, th);
            if (!P.visible) continue;
            const double* d = g2d + 9 * ((size_t)v * N + g);
            double gA = d[2], gB = d[3], gC = d[4];
            double a = P.a, b = P.b, c = P.c, det = P.det, det2 = det * det;
            /* conic (A, B, C) = (c, -b, a) / det  ->  (a, b, c) */
            double ga = gA * (-c * c / det2) + gB * (b * c / det2) + gC * (1.0 / det - a * c / det2);
            double gb = gA * (2.0 * b * c / det2) + gB * (-1.0 / det - 2.0 * b * b / det2) + gC * (2.0 * a * b / det2);
            double gc = gA * (1.0 / det - a * c / det2) + gB * (a * b / det2) + gC * (-a * a / det2);
            /* Sigma' = T Sigma T^T (+ dilation); symmetric gradient matrix */
            double G2[4] = {ga, 0.5 * gb, 0.5 * gb, gc};
            /* dL/dSigma += T^T G2 T */
            for (int i = 0; i < 3; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int p = 0; p < 2; p++)
                        for (int q = 0; q < 2; q++) acc += P.T[3 * p + i] * G2[2 * p + q] * P.T[3 * q + j];
                    gSig[3 * i + j] += acc;
                }
            /* dL/dT = 2 G2 T Sigma */
            double TS[6], gT[6], gJ[6];
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += P.T[3 * i + k] * G.Sig[3 * k + j];
                    TS[3 * i + j] = acc;
                }
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 3; j++) gT[3 * i + j] = 2.0 * (G2[2 * i] * TS[j] + G2[2 * i + 1] * TS[3 + j]);
            /* T = J Rc  ->  dL/dJ = dL/dT Rc^T */
            for (int i = 0; i < 2; i++)
                for (int j = 0; j < 3; j++) {
                    double acc = 0.0;
                    for (int k = 0; k < 3; k++) acc += gT[3 * i + k] * cam.R[3 * j + k];
                    gJ[3 * i + j] = acc;
                }
            double tx = P.t[0], ty = P.t[1], tz = P.t[2];
            double fx = cam.fx, fy = cam.fy;
            double gt[3] = {0, 0, 0};
            gt[2] += gJ[0] * (-fx / (tz * tz)) + gJ[4] * (-fy / (tz * tz));
            if (P.clx == 0) {
                gt[0] += gJ[2] * (-fx / (tz * tz));
                gt[2] += gJ[2] * (2.0 * fx * tx / (tz * tz * tz));
            } else {
                /* J02 = -fx * (+-lim) / tz */
                double lim = P.tc[0] / tz;
                gt[2] += gJ[2] * (fx * lim / (tz * tz));
            }
            if (P.cly == 0) {
                gt[1] += gJ[5] * (-fy / (tz * tz));
                gt[2] += gJ[5] * (2.0 * fy * ty / (tz * tz * tz));
            } else {
                double lim = P.tc[1] / tz;
                gt[2] += gJ[5] * (fy * lim / (tz * tz));
            }
            /* mean2d = (fx tx / tz + cx, fy ty / tz + cy) */
            gt[0] += d[0] * fx / tz;
            gt[1] += d[1] * fy / tz;
            gt[2] += -d[0] * fx * tx / (tz * tz) - d[1] * fy * ty / (tz * tz);
            /* t = Rc mu + tc */
            for (int j = 0; j < 3; j++) gmu[j] += cam.R[j] * gt[0] + cam.R[3 + j] * gt[1] + cam.R[6 + j] * gt[2];
            /* colour */
            double grgb[3];
            for (int ch = 0; ch < 3; ch++) grgb[ch] = (P.clampmask >> ch) & 1 ? 0.0 : d[6 + ch];
            double Y[16], dY[16][3];
            sh_eval(deg, P.dir[0], P.dir[1], P.dir[2], Y, dY);
            double gdir[3] = {0, 0, 0};
            for (int k = 0; k < nk; k++) {
                double w = 0.0;
                for (int ch = 0; ch < 3; ch++) {
                    gsh[3 * k + ch] += Y[k] * grgb[ch];
                    w += (double)shg[3 * k + ch] * grgb[ch];
                }
                for (int j = 0; j < 3; j++) gdir[j] += dY[k][j] * w;
            }
            double dd = gdir[0] * P.dir[0] + gdir[1] * P.dir[1] + gdir[2] * P.dir[2];
            for (int j = 0; j < 3; j++) gmu[j] += (gdir[j] - P.dir[j] * dd) / P.dlen;
            go += d[5];
        }
        for (int j = 0; j < 3; j++) g_means[3 * g + j] = gmu[j];
        g_logits[g] = go * G.o * (1.0 - G.o);
        /* Sigma = M M^T, M = R diag(s): dL/dM = 2 dL/dSigma M (dL/dSigma symmetric) */
        double gM[9];
        for (int i = 0; i < 3; i++)
            for (int j = 0; j < 3; j++) {
                double acc = 0.0;
                for (int k = 0; k < 3; k++) acc += (gSig[3 * i + k] + gSig[3 * k + i]) * G.M[3 * k + j];
                gM[3 * i + j] = acc;
            }
        double gR[9];
        for (int j = 0; j < 3; j++) {
            double acc = 0.0;
            for (int i = 0; i < 3; i++) {
                acc += gM[3 * i + j] * G.R[3 * i + j];
                gR[3 * i + j] = gM[3 * i + j] * G.s[j];
            }
            g_log_scales[3 * g + j] = acc * G.s[j];
        }
        double w = G.qn[0], x = G.qn[1], y = G.qn[2], z = G.qn[3];
        double gq[4];
        gq[0] = gR[1] * (-2 * z) + gR[2] * (2 * y) + gR[3] * (2 * z) + gR[5] * (-2 * x) + gR[6] * (-2 * y) + gR[7] * (2 * x);
        gq[1] = gR[1] * (2 * y) + gR[2] * (2 * z) + gR[3] * (2 * y) + gR[4] * (-4 * x) + gR[5] * (-2 * w) +
                gR[6] * (2 * z) + gR[7] * (2 * w) + gR[8] * (-4 * x);
        gq[2] = gR[0] * (-4 * y) + gR[1] * (2 * x) + gR[2] * (2 * w) + gR[3] * (2 * x) + gR[5] * (2 * z) +
                gR[6] * (-2 * w) + gR[7] * (2 * z) + gR[8] * (-4 * y);
        gq[3] = gR[0] * (-4 * z) + gR[1] * (-2 * w) + gR[2] * (2 * x) + gR[3] * (2 * w) + gR[4] * (-4 * z) +
                gR[5] * (2 * y) + gR[6] * (2 * x) + gR[7] * (2 * y);
        double dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
        for (int j = 0; j < 4; j++) g_quats[4 * g + j] = (gq[j] - G.qn[j] * dot) / G.qnorm;
    }
}
