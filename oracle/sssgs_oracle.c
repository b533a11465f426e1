/*
 * FP64 CPU oracle for the SSS Gaussian-splatting OLAT render.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares
 * no code, header or table with the CUDA path.
 *
 * Everything here is the plain definition, written for a reader to check
 * against the paper by eye:
 *   - EWA projection (Section 3.1 "3D Gaussian Splatting", Eq. 1, Eq. 2, and
 *     the scale/quaternion parameterisation of the covariance).
 *   - Front-to-back alpha compositing of every per-Gaussian property into an
 *     image-space buffer (Eq. 3; Fig. 2 caption; "Per-Pixel Deferred Shading").
 *   - Deferred BRDF shading per pixel (Eq. 4) blended with the SSS residual
 *     (Eq. 7), for one point light (Section 3.2 "Incident Light", OLAT).
 *   - Hand-derived backward of all of the above.
 *
 * Conventions the paper leaves open (each is a parameter or a fixed rule):
 *   alpha = min(alpha_max, o * exp(-p)), skipped when p < 0 or alpha < alpha_min;
 *   compositing stops before the Gaussian that would bring T below T_min;
 *   Gaussians are ordered by the float32 view-space depth, computed by the
 *   fused chain fmaf(R20, mx, fmaf(R21, my, fmaf(R22, mz, t2))), ties by index.
 *   Both sides take this ordering decision in float32, so orders agree exactly.
 *
 * Layouts (all double unless noted):
 *   cam[18]  = R (3x3 row-major, world->camera), t[3], fx, fy, cx, cy, W, H
 *   light[3] = point light position
 *   cfg[8]   = tile, dilation, det_eps, z_near, alpha_min, alpha_max, T_min, A_eps
 *   proj[N*16] = mx, my, ca, cb, cc, o, depth, L, ex, ey, tx, ty, tz, a, b, c
 *              (conic (ca,cb,cc) with p = 0.5*(ca dx^2 + cc dy^2) + cb dx dy,
 *               L = ln(o / alpha_min), AABB half extents ex, ey,
 *               dilated 2D covariance (a, b, c))
 *   rect[N*4]  = pixel bounds i0, i1, j0, j1 (inclusive); i0 > i1 => culled
 *   feat[N*15] = depth, n(3), base(3), rough, metal, sss, Lsss(3), Lin, vis
 *   gbuf[P*16] = sum_i w_i feat_i (15 channels) and final transmittance T
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NF 15
#define PI_D 3.14159265358979323846

/* ------------------------------------------------------------------ */
/* Projection (Eq. 1, Eq. 2)                                           */
/* ------------------------------------------------------------------ */

/* Rotation matrix of the unit quaternion (w, x, y, z). */
static void quat_to_rot(const double q[4], double R[9]) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Float32 depth key: the ordering decision both sides take in float32. */
float orc_depth_key_f32(const float Rc[9], const float tc[3], const float m[3]) {
    return fmaf(Rc[6], m[0], fmaf(Rc[7], m[1], fmaf(Rc[8], m[2], tc[2])));
}

static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* Sigma = R S S^T R^T with S = diag(exp(log_s)) and R from the normalised q. */
void orc_covariance(const double* log_s, const double* quat, double Sig[9]) {
    double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double q[4] = {quat[0] / qn, quat[1] / qn, quat[2] / qn, quat[3] / qn};
    double R[9];
    quat_to_rot(q, R);
    double s[3] = {exp(log_s[0]), exp(log_s[1]), exp(log_s[2])};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[i * 3 + k] * s[k] * s[k] * R[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }
}

int orc_project(int N, const double* mu, const double* log_s, const double* quat,
                const double* logit_o, const double* cam, const double* cfg,
                double* proj, int* rect, uint32_t* dkey) {
    const double* Rc = cam;
    const double* tc = cam + 9;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    int W = (int)cam[16], H = (int)cam[17];
    double dil = cfg[1], det_eps = cfg[2], z_near = cfg[3], a_min = cfg[4];
    float Rf[9], tf[3];
    for (int k = 0; k < 9; ++k) Rf[k] = (float)Rc[k];
    for (int k = 0; k < 3; ++k) tf[k] = (float)tc[k];
    for (int g = 0; g < N; ++g) {
        double* P = proj + 16 * (size_t)g;
        int* rc = rect + 4 * (size_t)g;
        memset(P, 0, 16 * sizeof(double));
        rc[0] = 1; rc[1] = 0; rc[2] = 1; rc[3] = 0;
        const double* m = mu + 3 * (size_t)g;
        float mf[3] = {(float)m[0], (float)m[1], (float)m[2]};
        float zk = orc_depth_key_f32(Rf, tf, mf);
        dkey[g] = f32_bits(zk);
        /* t = W mu + t_cam (view transform W of Eq. 2) */
        double t[3];
        for (int i = 0; i < 3; ++i)
            t[i] = Rc[i * 3 + 0] * m[0] + Rc[i * 3 + 1] * m[1] + Rc[i * 3 + 2] * m[2] + tc[i];
        P[10] = t[0]; P[11] = t[1]; P[12] = t[2];
        P[6] = t[2];
        double o = 1.0 / (1.0 + exp(-logit_o[g]));
        P[5] = o;
        if (t[2] < z_near) continue;
        double Sig[9];
        orc_covariance(log_s + 3 * (size_t)g, quat + 4 * (size_t)g, Sig);
        /* J: Jacobian of the affine approximation of the projection (Eq. 2) */
        double J[6] = {fx / t[2], 0, -fx * t[0] / (t[2] * t[2]),
                       0, fy / t[2], -fy * t[1] / (t[2] * t[2])};
        double T[6];  /* T = J W */
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[i * 3 + j] = J[i * 3 + 0] * Rc[0 * 3 + j] + J[i * 3 + 1] * Rc[1 * 3 + j] + J[i * 3 + 2] * Rc[2 * 3 + j];
        double S2[4];  /* Sigma' = T Sigma T^T */
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += T[i * 3 + k] * Sig[k * 3 + l] * T[j * 3 + l];
                S2[i * 2 + j] = acc;
            }
        double a = S2[0] + dil, b = S2[1], c = S2[3] + dil;
        P[13] = a; P[14] = b; P[15] = c;
        double det = a * c - b * b;
        if (det <= det_eps) continue;
        P[0] = fx * t[0] / t[2] + cx;
        P[1] = fy * t[1] / t[2] + cy;
        P[2] = c / det; P[3] = -b / det; P[4] = a / det;
        double L = log(o / a_min);
        P[7] = L;
        if (!(L > 0)) continue;
        /* alpha >= alpha_min  <=>  p <= L : the AABB of that ellipse */
        double ex = sqrt(2.0 * L * a) * (1.0 + 1e-9);
        double ey = sqrt(2.0 * L * c) * (1.0 + 1e-9);
        P[8] = ex; P[9] = ey;
        int i0 = (int)ceil(P[0] - ex - 0.5), i1 = (int)floor(P[0] + ex - 0.5);
        int j0 = (int)ceil(P[1] - ey - 0.5), j1 = (int)floor(P[1] + ey - 0.5);
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > W - 1) i1 = W - 1;
        if (j1 > H - 1) j1 = H - 1;
        if (i0 > i1 || j0 > j1) continue;
        rc[0] = i0; rc[1] = i1; rc[2] = j0; rc[3] = j1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Deferred shading (Eq. 4, Eq. 7)                                     */
/* ------------------------------------------------------------------ */

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Cook-Torrance specular with GGX D, Schlick F and separable Smith-GGX in
 * visibility form V = G / (4 no ni); Lambert diffuse (1 - m) b / pi.
 * Exposed for closed-form tests. */
void orc_brdf(const double* n, const double* wo, const double* wi, const double* base,
              double rough, double metal, double* fs, double* fd) {
    double H[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double hn = sqrt(dot3(H, H));
    double h[3] = {H[0] / hn, H[1] / hn, H[2] / hn};
    double no = fmax(dot3(n, wo), 0), ni = fmax(dot3(n, wi), 0);
    double nh = fmax(dot3(n, h), 0), vh = fmax(dot3(wo, h), 0);
    double ar = rough * rough, a2 = ar * ar;
    double den = nh * nh * (a2 - 1) + 1;
    double D = a2 / (PI_D * den * den);
    double V = 1.0 / ((no + sqrt(a2 + (1 - a2) * no * no)) * (ni + sqrt(a2 + (1 - a2) * ni * ni)));
    double w5 = pow(1 - vh, 5);
    for (int c = 0; c < 3; ++c) {
        double F0 = 0.04 * (1 - metal) + base[c] * metal;
        double Fr = F0 + (1 - F0) * w5;
        fs[c] = D * Fr * V;
        fd[c] = (1 - metal) * base[c] / PI_D;
    }
}

/* Forward shade of one pixel. F: composited features, T: final transmittance,
 * (u, v): pixel centre. Writes out[3]. If g3 != NULL also runs the backward
 * for upstream gradient g3 = dLoss/dout, writing dF[15] and *dT. */
static void shade_pixel(const double* F, double T, int has, double u, double v,
                        const double* cam, const double* light, double A_eps,
                        double* out, const double* g3, double* dF, double* dT) {
    out[0] = out[1] = out[2] = 0;
    if (g3) { memset(dF, 0, NF * sizeof(double)); *dT = 0; }
    if (!has) return;
    const double* R = cam;
    const double* t = cam + 9;
    double fx = cam[12], fy = cam[13], cx = cam[14], cy = cam[15];
    double A = 1.0 - T;
    double Ad = fmax(A, A_eps);
    double g[NF];
    for (int k = 0; k < NF; ++k) g[k] = F[k] / Ad;
    double dbar = g[0], rb = g[7], mb = g[8], sb = g[9], Li = g[13];
    const double* nbar = g + 1;
    const double* bb = g + 4;
    const double* Ls = g + 10;
    /* back-projected surface point x = R^T (d * ray - t) */
    double ray[3] = {(u - cx) / fx, (v - cy) / fy, 1.0};
    double Xc[3] = {dbar * ray[0] - t[0], dbar * ray[1] - t[1], dbar * ray[2] - t[2]};
    double x[3], C[3];
    for (int i = 0; i < 3; ++i) {
        x[i] = R[0 * 3 + i] * Xc[0] + R[1 * 3 + i] * Xc[1] + R[2 * 3 + i] * Xc[2];
        C[i] = -(R[0 * 3 + i] * t[0] + R[1 * 3 + i] * t[1] + R[2 * 3 + i] * t[2]);
    }
    double Vo[3] = {C[0] - x[0], C[1] - x[1], C[2] - x[2]};
    double Vi[3] = {light[0] - x[0], light[1] - x[1], light[2] - x[2]};
    double lo = sqrt(dot3(Vo, Vo)), li = sqrt(dot3(Vi, Vi));
    double wo[3] = {Vo[0] / lo, Vo[1] / lo, Vo[2] / lo};
    double wi[3] = {Vi[0] / li, Vi[1] / li, Vi[2] / li};
    double nn = sqrt(dot3(nbar, nbar));
    if (nn < 1e-12) nn = 1e-12;
    double nh_[3] = {nbar[0] / nn, nbar[1] / nn, nbar[2] / nn};
    double Hv[3] = {wo[0] + wi[0], wo[1] + wi[1], wo[2] + wi[2]};
    double lh = sqrt(dot3(Hv, Hv));
    double h[3] = {Hv[0] / lh, Hv[1] / lh, Hv[2] / lh};
    double co = dot3(nh_, wo), ci = dot3(nh_, wi), ch = dot3(nh_, h), cv = dot3(wo, h);
    double no = fmax(co, 0), ni = fmax(ci, 0), nh = fmax(ch, 0), vh = fmax(cv, 0);
    double ar = rb * rb, a2 = ar * ar;
    double den = nh * nh * (a2 - 1) + 1;
    double D = a2 / (PI_D * den * den);
    double so = sqrt(a2 + (1 - a2) * no * no), si = sqrt(a2 + (1 - a2) * ni * ni);
    double Lo = no + so, Lam_i = ni + si;
    double Vis = 1.0 / (Lo * Lam_i);
    double w5 = pow(1 - vh, 5);
    double F0[3], Fr[3], fs[3], fd[3], Lc[3];
    for (int c = 0; c < 3; ++c) {
        F0[c] = 0.04 * (1 - mb) + bb[c] * mb;
        Fr[c] = F0[c] + (1 - F0[c]) * w5;
        fs[c] = D * Fr[c] * Vis;
        fd[c] = (1 - mb) * bb[c] / PI_D;
        Lc[c] = sb * Ls[c] + (1 - sb) * (fs[c] + fd[c]) * Li * ni;
        out[c] = A * Lc[c];
    }
    if (!g3) return;

    /* ---- backward ---- */
    double dA = 0, dg[NF];
    memset(dg, 0, sizeof dg);
    double gL[3];
    for (int c = 0; c < 3; ++c) { dA += g3[c] * Lc[c]; gL[c] = g3[c] * A; }
    double dni = 0, dD = 0, dVis = 0, dw5 = 0, da2 = 0, dnh = 0, dvh = 0, dno = 0;
    for (int c = 0; c < 3; ++c) {
        dg[9] += gL[c] * (Ls[c] - (fs[c] + fd[c]) * Li * ni);
        dg[10 + c] += gL[c] * sb;
        dg[13] += gL[c] * (1 - sb) * (fs[c] + fd[c]) * ni;
        dni += gL[c] * (1 - sb) * (fs[c] + fd[c]) * Li;
        double cm = gL[c] * (1 - sb) * Li * ni;       /* d/d(fs + fd) */
        dg[8] += cm * (-bb[c] / PI_D);
        dg[4 + c] += cm * (1 - mb) / PI_D;
        dD += cm * Fr[c] * Vis;
        dVis += cm * D * Fr[c];
        double dFr = cm * D * Vis;
        double dF0 = dFr * (1 - w5);
        dw5 += dFr * (1 - F0[c]);
        dg[8] += dF0 * (bb[c] - 0.04);
        dg[4 + c] += dF0 * mb;
    }
    dvh += dw5 * (-5.0 * pow(1 - vh, 4));
    double dLo = -dVis * Vis / Lo, dLi = -dVis * Vis / Lam_i;
    dno += dLo * (1 + (1 - a2) * no / so);
    da2 += dLo * (1 - no * no) / (2 * so);
    dni += dLi * (1 + (1 - a2) * ni / si);
    da2 += dLi * (1 - ni * ni) / (2 * si);
    da2 += dD * (1.0 / (PI_D * den * den) - 2 * a2 * nh * nh / (PI_D * den * den * den));
    dnh += dD * (-4 * a2 * nh * (a2 - 1) / (PI_D * den * den * den));
    dg[7] += da2 * 4 * rb * rb * rb;
    double dco = co > 0 ? dno : 0, dci = ci > 0 ? dni : 0;
    double dch = ch > 0 ? dnh : 0, dcv = cv > 0 ? dvh : 0;
    double dn[3], dwo[3], dwi[3], dh[3];
    for (int i = 0; i < 3; ++i) {
        dn[i] = dco * wo[i] + dci * wi[i] + dch * h[i];
        dwo[i] = dco * nh_[i] + dcv * h[i];
        dwi[i] = dci * nh_[i];
        dh[i] = dch * nh_[i] + dcv * wo[i];
    }
    double hd = dot3(h, dh);
    for (int i = 0; i < 3; ++i) {
        double dH = (dh[i] - h[i] * hd) / lh;
        dwo[i] += dH; dwi[i] += dH;
    }
    double od = dot3(wo, dwo), id = dot3(wi, dwi), nd = dot3(nh_, dn);
    double dx[3];
    for (int i = 0; i < 3; ++i) {
        double dVo = (dwo[i] - wo[i] * od) / lo;
        double dVi = (dwi[i] - wi[i] * id) / li;
        dx[i] = -dVo - dVi;
        dg[1 + i] += (dn[i] - nh_[i] * nd) / nn;
    }
    /* x = R^T (d ray - t): dXc = R dx, d(dbar) = dXc . ray */
    double dXc[3];
    for (int i = 0; i < 3; ++i) dXc[i] = R[i * 3 + 0] * dx[0] + R[i * 3 + 1] * dx[1] + R[i * 3 + 2] * dx[2];
    dg[0] += dot3(dXc, ray);
    /* g = F / Ad */
    double dAd = 0;
    for (int k = 0; k < NF; ++k) { dF[k] = dg[k] / Ad; dAd -= dg[k] * g[k] / Ad; }
    if (A > A_eps) dA += dAd;
    *dT = -dA;
}

void orc_shade(int npix, const double* gbuf, const int* has, const int* pix,
               const double* cam, const double* light, const double* cfg,
               double* img, const double* dimg, double* dgbuf) {
    for (int q = 0; q < npix; ++q) {
        double u = pix[2 * q] + 0.5, v = pix[2 * q + 1] + 0.5;
        double dT;
        shade_pixel(gbuf + 16 * (size_t)q, gbuf[16 * (size_t)q + 15], has[q], u, v, cam, light, cfg[7],
                    img + 3 * (size_t)q, dimg ? dimg + 3 * (size_t)q : NULL,
                    dgbuf ? dgbuf + 16 * (size_t)q : NULL, &dT);
        if (dimg) dgbuf[16 * (size_t)q + 15] = dT;
    }
}

/* ------------------------------------------------------------------ */
/* Compositing (Eq. 3) and its backward                                */
/* ------------------------------------------------------------------ */

typedef struct { int g; double alpha, T, G; int clamped; } contrib_t;

static const uint32_t* g_sort_dkey;
static int cmp_depth(const void* a, const void* b) {
    int i = *(const int*)a, j = *(const int*)b;
    if (g_sort_dkey[i] != g_sort_dkey[j]) return g_sort_dkey[i] < g_sort_dkey[j] ? -1 : 1;
    return (i > j) - (i < j);
}

/*
 * Render one view/light pair. mode bit 0 clear: brute force (every valid
 * Gaussian is tested at every pixel, in depth order); set: tiled (each pixel
 * walks the depth-ordered list of Gaussians whose pixel rectangle touches its
 * tile). mode bit 1 set: per-Gaussian shading (the paper's "w/o Deferred"
 * ablation): feat[0..2] hold each Gaussian's own shaded colour and the image
 * is their composite (black background), img = F[0..2], dF = (dimg, 0, ...).
 * pix[npix*2] lists the pixels (i, j) to evaluate. Outputs per listed pixel:
 * gbuf[16], img[3], ncontrib, margin[3] (relative distance of the nearest
 * alpha decision and transmittance-stop decision to its threshold, and the
 * number of contributions whose alpha was clamped at alpha_max).
 * If dimg != NULL, accumulates per-Gaussian gradients into
 * dgeom[N*6] (dmx, dmy, dca, dcb, dcc, do) and dfeat[N*15].
 */
int orc_render(int N, const double* proj, const int* rect, const uint32_t* dkey,
               const double* feat, const double* cam, const double* light, const double* cfg,
               int mode, int npix, const int* pix,
               double* gbuf, double* img, int* ncontrib, double* margin,
               const double* dimg, double* dgeom, double* dfeat) {
    int tile = (int)cfg[0];
    const int tiled = mode & 1, per_gaussian = mode & 2;
    double a_min = cfg[4], a_max = cfg[5], T_min = cfg[6], A_eps = cfg[7];
    int W = (int)cam[16], H = (int)cam[17];
    int tiles_x = (W + tile - 1) / tile, tiles_y = (H + tile - 1) / tile;
    /* depth order of valid Gaussians */
    int* order = (int*)malloc(sizeof(int) * (size_t)(N > 0 ? N : 1));
    int nv = 0;
    for (int g = 0; g < N; ++g)
        if (rect[4 * g] <= rect[4 * g + 1]) order[nv++] = g;
        else if (!tiled && proj[16 * (size_t)g + 7] > 0 && proj[16 * (size_t)g + 12] >= cfg[3]) {
            /* brute force ignores rectangles; an off-screen Gaussian still has
             * no support at any pixel, so keep only ones that survive culling */
            double a = proj[16 * (size_t)g + 13], b = proj[16 * (size_t)g + 14], c = proj[16 * (size_t)g + 15];
            if (a * c - b * b > cfg[2]) order[nv++] = g;
        }
    g_sort_dkey = dkey;
    qsort(order, (size_t)nv, sizeof(int), cmp_depth);
    /* per-tile lists for tiled mode */
    int* tstart = NULL; int* tlist = NULL;
    if (tiled) {
        int nt = tiles_x * tiles_y;
        tstart = (int*)calloc((size_t)nt + 1, sizeof(int));
        for (int k = 0; k < nv; ++k) {
            const int* r = rect + 4 * order[k];
            for (int ty = r[2] / tile; ty <= r[3] / tile; ++ty)
                for (int tx = r[0] / tile; tx <= r[1] / tile; ++tx) tstart[ty * tiles_x + tx + 1]++;
        }
        for (int t = 0; t < nt; ++t) tstart[t + 1] += tstart[t];
        tlist = (int*)malloc(sizeof(int) * (size_t)(tstart[nt] > 0 ? tstart[nt] : 1));
        int* fill = (int*)malloc(sizeof(int) * (size_t)nt);
        memcpy(fill, tstart, sizeof(int) * (size_t)nt);
        for (int k = 0; k < nv; ++k) {
            const int* r = rect + 4 * order[k];
            for (int ty = r[2] / tile; ty <= r[3] / tile; ++ty)
                for (int tx = r[0] / tile; tx <= r[1] / tile; ++tx) tlist[fill[ty * tiles_x + tx]++] = order[k];
        }
        free(fill);
    }
    contrib_t* cb = (contrib_t*)malloc(sizeof(contrib_t) * (size_t)(nv > 0 ? nv : 1));
    for (int q = 0; q < npix; ++q) {
        int pi = pix[2 * q], pj = pix[2 * q + 1];
        double px = pi + 0.5, py = pj + 0.5;
        const int* list; int nl;
        if (tiled) {
            int t = (pj / tile) * tiles_x + pi / tile;
            list = tlist + tstart[t]; nl = tstart[t + 1] - tstart[t];
        } else { list = order; nl = nv; }
        double F[NF] = {0}, T = 1.0;
        double ma = INFINITY, mt = INFINITY;
        int nc = 0, ncl = 0;
        for (int k = 0; k < nl; ++k) {
            int g = list[k];
            const double* P = proj + 16 * (size_t)g;
            double dx = P[0] - px, dy = P[1] - py;
            double p = 0.5 * (P[2] * dx * dx + P[4] * dy * dy) + P[3] * dx * dy;
            if (p < 0) continue;
            double G = exp(-p);
            double araw = P[5] * G;
            ma = fmin(ma, fabs(araw - a_min) / a_min);
            ma = fmin(ma, fabs(araw - a_max) / a_max);
            double alpha = fmin(a_max, araw);
            if (alpha < a_min) continue;
            double Tn = T * (1 - alpha);
            mt = fmin(mt, fabs(Tn - T_min) / T_min);
            if (Tn < T_min) break;
            double w = T * alpha;
            const double* f = feat + NF * (size_t)g;
            for (int c = 0; c < NF; ++c) F[c] += w * f[c];
            cb[nc].g = g; cb[nc].alpha = alpha; cb[nc].T = T; cb[nc].G = G; cb[nc].clamped = araw > a_max;
            ncl += cb[nc].clamped;
            ++nc;
            T = Tn;
        }
        double* gb = gbuf + 16 * (size_t)q;
        for (int c = 0; c < NF; ++c) gb[c] = F[c];
        gb[15] = T;
        ncontrib[q] = nc;
        margin[3 * q] = ma; margin[3 * q + 1] = mt; margin[3 * q + 2] = ncl;
        double dF[NF], dT;
        if (per_gaussian) {
            for (int c = 0; c < 3; ++c) img[3 * (size_t)q + c] = F[c];
            memset(dF, 0, sizeof(dF));
            dT = 0;
            if (dimg) for (int c = 0; c < 3; ++c) dF[c] = dimg[3 * (size_t)q + c];
        } else {
            shade_pixel(F, T, nc > 0, px, py, cam, light, A_eps, img + 3 * (size_t)q,
                        dimg ? dimg + 3 * (size_t)q : NULL, dF, &dT);
        }
        if (!dimg || nc == 0) continue;
        /* dLoss/dalpha_i = sum_k dF_k (T_i f_ik - S_ik / (1 - alpha_i))
         *                  - dT * T_final / (1 - alpha_i),
         * S_ik = sum_{j>i} T_j alpha_j f_jk (plain derivative of Eq. 3). */
        double S[NF] = {0};
        for (int i = nc - 1; i >= 0; --i) {
            int g = cb[i].g;
            const double* f = feat + NF * (size_t)g;
            double a = cb[i].alpha, Ti = cb[i].T, w = Ti * a;
            double da = -dT * T / (1 - a);
            for (int c = 0; c < NF; ++c) da += dF[c] * (Ti * f[c] - S[c] / (1 - a));
            for (int c = 0; c < NF; ++c) {
                dfeat[NF * (size_t)g + c] += w * dF[c];
                S[c] += w * f[c];
            }
            if (cb[i].clamped) continue;
            const double* P = proj + 16 * (size_t)g;
            double dx = P[0] - px, dy = P[1] - py;
            double dp = -da * a;            /* alpha = o exp(-p) */
            double* dg = dgeom + 6 * (size_t)g;
            dg[5] += da * cb[i].G;
            dg[2] += dp * 0.5 * dx * dx;
            dg[3] += dp * dx * dy;
            dg[4] += dp * 0.5 * dy * dy;
            dg[0] += dp * (P[2] * dx + P[3] * dy);
            dg[1] += dp * (P[3] * dx + P[4] * dy);
        }
    }
    free(cb); free(order); free(tstart); free(tlist);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Projection backward                                                 */
/* ------------------------------------------------------------------ */

/* dgeom[N*6] (dmx, dmy, dca, dcb, dcc, do), ddepth[N] -> parameter grads
 * (accumulated into d_mu[N*3], d_log_s[N*3], d_quat[N*4], d_logit[N]). */
int orc_project_bwd(int N, const double* mu, const double* log_s, const double* quat,
                    const double* logit_o, const double* cam, const double* proj, const int* rect,
                    const double* dgeom, const double* ddepth,
                    double* d_mu, double* d_log_s, double* d_quat, double* d_logit) {
    const double* Rc = cam;
    double fx = cam[12], fy = cam[13];
    for (int g = 0; g < N; ++g) {
        if (rect[4 * g] > rect[4 * g + 1]) continue;   /* culled: no gradient */
        const double* P = proj + 16 * (size_t)g;
        const double* dg = dgeom + 6 * (size_t)g;
        double o = P[5];
        d_logit[g] += dg[5] * o * (1 - o);
        double tx = P[10], ty = P[11], tz = P[12];
        double dt[3] = {0, 0, 0};
        dt[0] += dg[0] * fx / tz;
        dt[1] += dg[1] * fy / tz;
        dt[2] += -dg[0] * fx * tx / (tz * tz) - dg[1] * fy * ty / (tz * tz);
        dt[2] += ddepth[g];
        /* conic = inverse(Sigma'):  dSigma' = -C Gbar C  (symmetric form) */
        double C[4] = {P[2], P[3], P[3], P[4]};
        double Gb[4] = {dg[2], 0.5 * dg[3], 0.5 * dg[3], dg[4]};
        double CG[4], Gs[4];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) CG[i * 2 + j] = C[i * 2 + 0] * Gb[0 * 2 + j] + C[i * 2 + 1] * Gb[1 * 2 + j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) Gs[i * 2 + j] = -(CG[i * 2 + 0] * C[0 * 2 + j] + CG[i * 2 + 1] * C[1 * 2 + j]);
        double J[6] = {fx / tz, 0, -fx * tx / (tz * tz), 0, fy / tz, -fy * ty / (tz * tz)};
        double T[6];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                T[i * 3 + j] = J[i * 3 + 0] * Rc[0 * 3 + j] + J[i * 3 + 1] * Rc[1 * 3 + j] + J[i * 3 + 2] * Rc[2 * 3 + j];
        double Sig[9];
        orc_covariance(log_s + 3 * (size_t)g, quat + 4 * (size_t)g, Sig);
        /* dT = 2 Gs T Sigma ; dJ = dT W^T ; dSigma = T^T Gs T */
        double GT[6], dT[6], dJ[6], dS[9];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) GT[i * 3 + j] = Gs[i * 2 + 0] * T[0 * 3 + j] + Gs[i * 2 + 1] * T[1 * 3 + j];
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += GT[i * 3 + k] * Sig[k * 3 + j];
                dT[i * 3 + j] = 2 * acc;
            }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 3; ++j)
                dJ[i * 3 + j] = dT[i * 3 + 0] * Rc[j * 3 + 0] + dT[i * 3 + 1] * Rc[j * 3 + 1] + dT[i * 3 + 2] * Rc[j * 3 + 2];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) dS[i * 3 + j] = T[0 * 3 + i] * GT[0 * 3 + j] + T[1 * 3 + i] * GT[1 * 3 + j];
        double tz2 = tz * tz, tz3 = tz2 * tz;
        dt[0] += dJ[2] * (-fx / tz2);
        dt[1] += dJ[5] * (-fy / tz2);
        dt[2] += dJ[0] * (-fx / tz2) + dJ[2] * (2 * fx * tx / tz3) + dJ[4] * (-fy / tz2) + dJ[5] * (2 * fy * ty / tz3);
        for (int i = 0; i < 3; ++i)
            d_mu[3 * (size_t)g + i] += Rc[0 * 3 + i] * dt[0] + Rc[1 * 3 + i] * dt[1] + Rc[2 * 3 + i] * dt[2];
        /* Sigma = M M^T, M = R S */
        const double* qq = quat + 4 * (size_t)g;
        double qn = sqrt(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
        double q[4] = {qq[0] / qn, qq[1] / qn, qq[2] / qn, qq[3] / qn};
        double R[9];
        quat_to_rot(q, R);
        const double* ls = log_s + 3 * (size_t)g;
        double s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};
        double M[9], dM[9], dR[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i * 3 + j] = R[i * 3 + j] * s[j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += dS[i * 3 + k] * M[k * 3 + j];
                dM[i * 3 + j] = 2 * acc;
            }
        for (int j = 0; j < 3; ++j) {
            double ds = 0;
            for (int i = 0; i < 3; ++i) { dR[i * 3 + j] = dM[i * 3 + j] * s[j]; ds += dM[i * 3 + j] * R[i * 3 + j]; }
            d_log_s[3 * (size_t)g + j] += ds * s[j];
        }
        double w = q[0], x = q[1], y = q[2], z = q[3];
        const double* G = dR;
        double dq[4];
        dq[0] = 2 * (-z * G[1] + y * G[2] + z * G[3] - x * G[5] - y * G[6] + x * G[7]);
        dq[1] = 2 * (y * G[1] + z * G[2] + y * G[3] - 2 * x * G[4] - w * G[5] + z * G[6] + w * G[7] - 2 * x * G[8]);
        dq[2] = 2 * (-2 * y * G[0] + x * G[1] + w * G[2] + x * G[3] + z * G[5] - w * G[6] + z * G[7] - 2 * y * G[8]);
        dq[3] = 2 * (-2 * z * G[0] - w * G[1] + x * G[2] + w * G[3] - 2 * z * G[4] + y * G[5] + x * G[6] + y * G[7]);
        double qd = q[0] * dq[0] + q[1] * dq[1] + q[2] * dq[2] + q[3] * dq[3];
        for (int k = 0; k < 4; ++k) d_quat[4 * (size_t)g + k] += (dq[k] - q[k] * qd) / qn;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Tile binning + depth ordering (plain stable sort of the definition) */
/* ------------------------------------------------------------------ */

typedef struct { uint32_t tile, dkey, item; } inst_t;
static int cmp_inst(const void* a, const void* b) {
    const inst_t* x = (const inst_t*)a; const inst_t* y = (const inst_t*)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->dkey != y->dkey) return x->dkey < y->dkey ? -1 : 1;
    return (x->item > y->item) - (x->item < y->item);
}

/*
 * Items are (pair, Gaussian) rows; item_pair[m] gives the pair, trect[m*4] the
 * inclusive tile rectangle (tx0, tx1, ty0, ty1; tx0 > tx1 = culled), dkey[m]
 * the float32 depth bits. Each pair p owns tiles [tile_off[p], tile_off[p] +
 * tiles_x[p] * tiles_y[p]). For every item and every tile of its rectangle one
 * instance (global tile, item) is emitted; instances are ordered by (tile,
 * depth key, item). Writes up to `capacity` of them and per-tile [start, end).
 * Returns the total number of instances.
 */
long long orc_bin(int n_items, const int* item_pair, const int* trect, const uint32_t* dkey,
                  const int* tiles_x, const int* tile_off, int total_tiles,
                  long long capacity, uint32_t* keys, uint32_t* vals, uint32_t* ranges) {
    long long n = 0;
    for (int m = 0; m < n_items; ++m) {
        const int* r = trect + 4 * (size_t)m;
        if (r[0] > r[1] || r[2] > r[3]) continue;
        n += (long long)(r[1] - r[0] + 1) * (r[3] - r[2] + 1);
    }
    inst_t* in = (inst_t*)malloc(sizeof(inst_t) * (size_t)(n > 0 ? n : 1));
    long long k = 0;
    for (int m = 0; m < n_items; ++m) {
        const int* r = trect + 4 * (size_t)m;
        if (r[0] > r[1] || r[2] > r[3]) continue;
        int p = item_pair[m];
        for (int ty = r[2]; ty <= r[3]; ++ty)
            for (int tx = r[0]; tx <= r[1]; ++tx) {
                in[k].tile = (uint32_t)(tile_off[p] + ty * tiles_x[p] + tx);
                in[k].dkey = dkey[m];
                in[k].item = (uint32_t)m;
                ++k;
            }
    }
    qsort(in, (size_t)n, sizeof(inst_t), cmp_inst);
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)total_tiles);
    for (long long i = 0; i < n && i < capacity; ++i) { keys[i] = in[i].tile; vals[i] = in[i].item; }
    for (long long i = 0; i < n; ++i) {
        uint32_t t = in[i].tile;
        if (i == 0 || in[i - 1].tile != t) ranges[2 * t] = (uint32_t)i;
        if (i == n - 1 || in[i + 1].tile != t) ranges[2 * t + 1] = (uint32_t)(i + 1);
    }
    free(in);
    return n;
}
