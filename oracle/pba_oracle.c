/*
 * FP64 CPU oracle for photometric bundle adjustment (PBA) in the inverse
 * compositional form with proxy templates (IC) and in the forwards
 * compositional form (FC), after Ham, Lucey and Singh, "Proxy Templates for
 * Inverse Compositional Photometric Bundle Adjustment", ICCV 2017
 * (arXiv 1704.06967).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow reference that the
 * GPU library is checked against. Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load it; the library never does. It shares
 * no code, header or table with the GPU path.
 *
 * Everything is double precision, single threaded, and written as the plain
 * loops of the definitions, in the paper's order and notation:
 *   Sec. 3 (Eq. energy, Eq. warp): residual r = I_0(x) - I_f(W(x; p_fn)),
 *      W(x;p) = <R x~ + d t>, one inverse depth d_n per point shared by its
 *      pattern pixels.
 *   Sec. 3 (Notation): bilinear image functions, <.> projection on z = 1,
 *      left-multiplicative pose update (the "boxplus" operator).
 *   Sec. 3.2-3.4 (Eq. phi, Eq. phi0, Eq. phi_grad, Eq. phi_update): the proxy
 *      warp phi and its partial derivatives at Delta p = 0.
 *   Sec. 3.5: J_nfx = grad I_0 dphi/dDelta p, H = J^T W_0 J with the initial
 *      Huber weights, the four-step Gauss-Newton loop.
 *   Sec. 3.6: inverse update composition (R, t, d update rules).
 * Readings of what the paper leaves open (all shared with the GPU library by
 * specification, not by code):
 *   - pixel coordinates u = f_x x + c_x (the paper works on the z = 1 plane);
 *   - image gradient = central differences at integer pixels; FC samples the
 *     gradient images bilinearly;
 *   - a residual is valid when the 2x2 bilinear footprint lies in
 *     [1, W-2] x [1, H-2] (so gradients exist) and the point is in front;
 *   - Huber: rho(r) = r^2/2 for |r| <= k else k|r| - k^2/2, IRLS weight
 *     w = min(1, k/|r|);
 *   - zbar_0 = [R_0 x~ + d_0 t_0]_z / d_0 (the proxy-image depth that makes
 *     phi(x;0) = x hold);
 *   - IC parameter order per frame [Delta t, omega] with R' = exp(omega) R_0,
 *     t' = t_0 + Delta t; FC order [upsilon, omega] with T <- exp(xi) T;
 *   - gauge: global scale is free; a prior mu * that^T that on the
 *     translation block of the first active target frame (that = unit t of
 *     that frame, p_0 for IC, current for FC; mu = mean diagonal of S) fixes
 *     it; frames without residuals get an identity block; points without
 *     residuals keep their depth;
 *   - IC keeps the residual set of p_0: a residual contributes to g only if
 *     it was valid at p_0 (else its stored J row is zero) and is valid now.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int W, H, F, N, P;
    double fx, fy, cx, cy, huber_k;
    const double* img;          /* F*H*W intensities, frame-major, row-major */
    const int* uv;              /* N*2 integer pixel centres in frame 0 */
    const int* pat;             /* P*2 pattern offsets (pixels) */
    const unsigned char* vis;   /* N*F visibility, vis[n*F+f] */
    double damping;             /* Levenberg-Marquardt lambda (0: Gauss-Newton) */
    double* photo;              /* F*2 affine brightness (alpha_f, beta_f) or NULL (model off) */
    double photo_prior;         /* joint brightness step: prior weight lambda >= 0 (0: none) */
} or_problem;

/* IC precompute (Sec. 3.5), indexed by residual id ((n*F + f)*P + j). */
typedef struct {
    double* J;                  /* R*7: [dt(3), omega(3), dd] */
    double* r0;                 /* R */
    double* w0;                 /* R */
    unsigned char* valid0;      /* R */
    double* Hff;                /* F*36, frame 0 block unused (zero) */
    double* Hfd;                /* N*F*6 */
    double* Hdd;                /* N */
} or_ic_pre;

enum { OR_OK = 0, OR_ERR_NOT_PD = 5 };

/* ------------------------------------------------------------------------ */
/* small linear algebra                                                      */
/* ------------------------------------------------------------------------ */
static void mat3_mul(const double* A, const double* B, double* C)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = s;
        }
    memcpy(C, T, sizeof T);
}

static void mat3_transpose(const double* A, double* B)
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) T[3 * i + j] = A[3 * j + i];
    memcpy(B, T, sizeof T);
}

static void mat3_vec(const double* A, const double* v, double* out)
{
    double o[3];
    for (int i = 0; i < 3; ++i) o[i] = A[3 * i] * v[0] + A[3 * i + 1] * v[1] + A[3 * i + 2] * v[2];
    memcpy(out, o, sizeof o);
}

static void skew(const double* a, double* S)
{
    S[0] = 0.0;   S[1] = -a[2]; S[2] = a[1];
    S[3] = a[2];  S[4] = 0.0;   S[5] = -a[0];
    S[6] = -a[1]; S[7] = a[0];  S[8] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* Lie groups (Sec. 1 / Sec. 3 Notation: T = exp(theta))                     */
/* ------------------------------------------------------------------------ */
/* SO(3) exp by Rodrigues' formula R = I + A [w]x + B [w]x^2 with
 * A = sin(th)/th, B = (1-cos(th))/th^2; Taylor series below th = 1e-3. */
void or_so3_exp(const double* w, double* R)
{
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B;
    if (th < 1e-3) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
    } else {
        A = sin(th) / th;
        B = (1.0 - cos(th)) / th2;
    }
    double K[9], K2[9];
    skew(w, K);
    mat3_mul(K, K, K2);
    for (int i = 0; i < 9; ++i) R[i] = A * K[i] + B * K2[i];
    R[0] += 1.0; R[4] += 1.0; R[8] += 1.0;
}

/* SE(3) exp of xi = [upsilon, omega]: R = exp(omega), t = V upsilon with
 * V = I + B [w]x + C [w]x^2, C = (th - sin th)/th^3 (Taylor below 1e-3). */
void or_se3_exp(const double* xi, double* R, double* t)
{
    const double* v = xi;
    const double* w = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double B, C;
    if (th < 1e-3) {
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        C = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        B = (1.0 - cos(th)) / th2;
        C = (th - sin(th)) / (th2 * th);
    }
    or_so3_exp(w, R);
    double K[9], K2[9], V[9];
    skew(w, K);
    mat3_mul(K, K, K2);
    for (int i = 0; i < 9; ++i) V[i] = B * K[i] + C * K2[i];
    V[0] += 1.0; V[4] += 1.0; V[8] += 1.0;
    mat3_vec(V, v, t);
}

/* ------------------------------------------------------------------------ */
/* images (Sec. 3 Notation: functions over images are bilinear)              */
/* ------------------------------------------------------------------------ */
static double pix(const double* img, int W, int x, int y) { return img[(size_t)y * W + x]; }

/* Bilinear I(u,v) at pixel coordinates (pixel centres on integers). Valid iff
 * the 2x2 footprint lies in [1, W-2] x [1, H-2]. Returns 1 when valid. */
int or_bilinear(const double* img, int W, int H, double u, double v, double* out)
{
    double fu = floor(u), fv = floor(v);
    if (!(fu >= 1.0 && fu + 1.0 <= W - 2 && fv >= 1.0 && fv + 1.0 <= H - 2)) {
        *out = 0.0;
        return 0;
    }
    int x = (int)fu, y = (int)fv;
    double a = u - fu, b = v - fv;
    *out = (1.0 - a) * (1.0 - b) * pix(img, W, x, y) + a * (1.0 - b) * pix(img, W, x + 1, y)
         + (1.0 - a) * b * pix(img, W, x, y + 1) + a * b * pix(img, W, x + 1, y + 1);
    return 1;
}

/* Central-difference gradient at an integer pixel, 1 <= x <= W-2. */
void or_grad_central(const double* img, int W, int H, int x, int y, double* gu, double* gv)
{
    (void)H;
    *gu = 0.5 * (pix(img, W, x + 1, y) - pix(img, W, x - 1, y));
    *gv = 0.5 * (pix(img, W, x, y + 1) - pix(img, W, x, y - 1));
}

/* Bilinear sample of the central-difference gradient images (FC). */
static void grad_bilinear(const double* img, int W, double u, double v, double* gu, double* gv)
{
    int x = (int)floor(u), y = (int)floor(v);
    double a = u - x, b = v - y;
    double w00 = (1 - a) * (1 - b), w10 = a * (1 - b), w01 = (1 - a) * b, w11 = a * b;
    double g[4][2];
    int xs[4] = {x, x + 1, x, x + 1}, ys[4] = {y, y, y + 1, y + 1};
    for (int i = 0; i < 4; ++i) or_grad_central(img, W, 0, xs[i], ys[i], &g[i][0], &g[i][1]);
    *gu = w00 * g[0][0] + w10 * g[1][0] + w01 * g[2][0] + w11 * g[3][0];
    *gv = w00 * g[0][1] + w10 * g[1][1] + w01 * g[2][1] + w11 * g[3][1];
}

/* ------------------------------------------------------------------------ */
/* warps                                                                     */
/* ------------------------------------------------------------------------ */
/* Eq. warp: W(x;p) = <R x~ + d t>. Returns the 3-vector q = R x~ + d t in q
 * and its projection in out (normalised coordinates). Returns q_z > 0. */
int or_warp(const double* R, const double* t, double d, double x, double y, double* out,
            double* q)
{
    double xt[3] = {x, y, 1.0}, qq[3];
    mat3_vec(R, xt, qq);
    for (int i = 0; i < 3; ++i) qq[i] += d * t[i];
    if (q) memcpy(q, qq, sizeof qq);
    out[0] = qq[0] / qq[2];
    out[1] = qq[1] / qq[2];
    return qq[2] > 0.0;
}

/* Eq. phi0: phi(x;dp) = W(W(x; dp (+) p0); p0)^-1, with the inverse warp of
 * p0 taken at the proxy depth zbar_0 = [R0 x~ + d0 t0]_z / d0:
 *   phi = < R0^T ( zbar_0 * W~(x; p') - t0 ) >,
 * p' = (R' = exp(omega) R0, t' = t0 + dt, d' = d0 + dd), dp = [dt, omega, dd]. */
void or_phi(const double* R0, const double* t0, double d0, double x, double y,
            const double* dp, double* out)
{
    double xt[3] = {x, y, 1.0}, v0[3];
    mat3_vec(R0, xt, v0);
    for (int i = 0; i < 3; ++i) v0[i] += d0 * t0[i];
    double zbar0 = v0[2] / d0;
    double dR[9], Rp[9], tp[3];
    or_so3_exp(dp + 3, dR);
    mat3_mul(dR, R0, Rp);
    for (int i = 0; i < 3; ++i) tp[i] = t0[i] + dp[i];
    double dprime = d0 + dp[6];
    double w[2], q[3];
    or_warp(Rp, tp, dprime, x, y, w, q);
    double yt[3] = {w[0], w[1], 1.0}, X[3], R0t[9];
    for (int i = 0; i < 3; ++i) X[i] = zbar0 * yt[i] - t0[i];
    mat3_transpose(R0, R0t);
    mat3_vec(R0t, X, X);
    out[0] = X[0] / X[2];
    out[1] = X[1] / X[2];
}

/* Eq. phi_update (small-update form used to derive the warp update):
 *   phi ~= < R0^T ( (1/d') R' x~ + dt ) >. */
void or_phi_update(const double* R0, const double* t0, double d0, double x, double y,
                   const double* dp, double* out)
{
    (void)t0;
    double xt[3] = {x, y, 1.0}, dR[9], Rp[9], a[3], R0t[9];
    or_so3_exp(dp + 3, dR);
    mat3_mul(dR, R0, Rp);
    mat3_vec(Rp, xt, a);
    double dprime = d0 + dp[6];
    for (int i = 0; i < 3; ++i) a[i] = a[i] / dprime + dp[i];
    mat3_transpose(R0, R0t);
    mat3_vec(R0t, a, a);
    out[0] = a[0] / a[2];
    out[1] = a[1] / a[2];
}

/* Sec. 3.4: dphi/d(dp) at dp = 0 in normalised coordinates (2x7, row-major).
 *   M = R0^T (zbar_0 I - [0 0 t0]),  phi* = M (R' x~ + d' t'),
 *   dphi* / d dt = d0 M, dphi* / d omega = -M [R0 x~]x, dphi* / d dd = M t0,
 *   quotient rule at v = phi*(x;0):  d<v> = (1/v_z^2) [dv_x v_z - v_x dv_z; ...]. */
void or_phi_jacobian(const double* R0, const double* t0, double d0, double x, double y,
                     double* Jphi)
{
    double xt[3] = {x, y, 1.0}, a[3], v0[3];
    mat3_vec(R0, xt, a);                        /* R0 x~ */
    for (int i = 0; i < 3; ++i) v0[i] = a[i] + d0 * t0[i];
    double zbar0 = v0[2] / d0;
    double inner[9] = {zbar0, 0, -t0[0], 0, zbar0, -t0[1], 0, 0, zbar0 - t0[2]};
    double R0t[9], M[9];
    mat3_transpose(R0, R0t);
    mat3_mul(R0t, inner, M);
    double dstar[3][7];                         /* dphi* / d(dp), 3x7 */
    double Sa[9], MSa[9], Mt0[3];
    skew(a, Sa);
    mat3_mul(M, Sa, MSa);
    mat3_vec(M, t0, Mt0);
    for (int i = 0; i < 3; ++i) {
        for (int k = 0; k < 3; ++k) {
            dstar[i][k] = d0 * M[3 * i + k];
            dstar[i][3 + k] = -MSa[3 * i + k];
        }
        dstar[i][6] = Mt0[i];
    }
    double v[3];
    mat3_vec(M, v0, v);                         /* phi*(x; 0) */
    for (int k = 0; k < 7; ++k) {
        Jphi[k] = (dstar[0][k] * v[2] - v[0] * dstar[2][k]) / (v[2] * v[2]);
        Jphi[7 + k] = (dstar[1][k] * v[2] - v[1] * dstar[2][k]) / (v[2] * v[2]);
    }
}

/* ------------------------------------------------------------------------ */
/* Huber (Eq. energy, ||.||_gamma)                                           */
/* ------------------------------------------------------------------------ */
double or_huber_rho(double r, double k)
{
    double a = fabs(r);
    return a <= k ? 0.5 * r * r : k * a - 0.5 * k * k;
}

double or_huber_weight(double r, double k)
{
    double a = fabs(r);
    return a <= k ? 1.0 : k / a;
}

/* ------------------------------------------------------------------------ */
/* residual geometry                                                         */
/* ------------------------------------------------------------------------ */
static const double* frame_img(const or_problem* pb, int f)
{
    return pb->img + (size_t)f * pb->H * pb->W;
}

/* normalised coordinates and integer pixel of pattern pixel j of point n */
static void pattern_pixel(const or_problem* pb, int n, int j, int* px, int* py, double* x,
                          double* y)
{
    *px = pb->uv[2 * n] + pb->pat[2 * j];
    *py = pb->uv[2 * n + 1] + pb->pat[2 * j + 1];
    *x = (*px - pb->cx) / pb->fx;
    *y = (*py - pb->cy) / pb->fy;
}

/* Residual r = I_0(x) - I_f(W(x; p_fn)) (Sec. 3.5) at pose (R,t), depth d.
 * Returns validity; fills pixel position u[2] and q = R x~ + d t. */
static int residual_at(const or_problem* pb, int n, int f, int j, const double* R,
                       const double* t, double d, double* r, double* u, double* q)
{
    int px, py;
    double x, y, w[2];
    pattern_pixel(pb, n, j, &px, &py, &x, &y);
    int front = or_warp(R, t, d, x, y, w, q);
    u[0] = pb->fx * w[0] + pb->cx;
    u[1] = pb->fy * w[1] + pb->cy;
    double If;
    if (!front || !or_bilinear(frame_img(pb, f), pb->W, pb->H, u[0], u[1], &If)) {
        *r = 0.0;
        return 0;
    }
    /* affine brightness of frame f: the template sees alpha_f I_f + beta_f */
    if (pb->photo) If = pb->photo[2 * f] * If + pb->photo[2 * f + 1];
    *r = pix(frame_img(pb, 0), pb->W, px, py) - If;
    return 1;
}

/* One IC residual at p0 (Sec. 3.5): J row = grad I_0(x) * dphi/d(dp),
 * with the pixel chain rule [g_u f_x, g_v f_y]; r0 and validity at p0. */
int or_ic_residual(const or_problem* pb, const double* poses0, const double* depths0, int n,
                   int f, int j, double* Jrow, double* r0)
{
    const double* R0 = poses0 + 12 * f;
    const double* t0 = R0 + 9;
    double d0 = depths0[n];
    double u[2], q[3];
    int valid = residual_at(pb, n, f, j, R0, t0, d0, r0, u, q);
    int px, py;
    double x, y, gu, gv, Jphi[14];
    pattern_pixel(pb, n, j, &px, &py, &x, &y);
    or_grad_central(frame_img(pb, 0), pb->W, pb->H, px, py, &gu, &gv);
    or_phi_jacobian(R0, t0, d0, x, y, Jphi);
    for (int k = 0; k < 7; ++k) Jrow[k] = gu * pb->fx * Jphi[k] + gv * pb->fy * Jphi[7 + k];
    return valid;
}

/* One FC residual at the current p: r and J = dr/d(dp) for the left update
 * T <- exp([upsilon, omega]) T, d <- d + dd:
 *   dq/dupsilon = d I, dq/domega = -[q]x, dq/dd = t,
 *   J = -[g_u f_x, g_v f_y] (1/q_z) [[1,0,-q_x/q_z],[0,1,-q_y/q_z]] dq/d(dp). */
int or_fc_residual(const or_problem* pb, const double* poses, const double* depths, int n,
                   int f, int j, double* Jrow, double* r)
{
    const double* R = poses + 12 * f;
    const double* t = R + 9;
    double d = depths[n];
    double u[2], q[3];
    int valid = residual_at(pb, n, f, j, R, t, d, r, u, q);
    for (int k = 0; k < 7; ++k) Jrow[k] = 0.0;
    if (!valid) return 0;
    double gu, gv;
    grad_bilinear(frame_img(pb, f), pb->W, u[0], u[1], &gu, &gv);
    double dq[3][7] = {{0}};
    double Sq[9];
    skew(q, Sq);
    for (int i = 0; i < 3; ++i) {
        dq[i][i] = d;
        for (int k = 0; k < 3; ++k) dq[i][3 + k] = -Sq[3 * i + k];
        dq[i][6] = t[i];
    }
    double iz = 1.0 / q[2];
    const double alpha = pb->photo ? pb->photo[2 * f] : 1.0;
    for (int k = 0; k < 7; ++k) {
        double dx = iz * (dq[0][k] - q[0] * iz * dq[2][k]);
        double dy = iz * (dq[1][k] - q[1] * iz * dq[2][k]);
        Jrow[k] = -alpha * (gu * pb->fx * dx + gv * pb->fy * dy);
    }
    return 1;
}

static size_t rid(const or_problem* pb, int n, int f, int j)
{
    return ((size_t)n * pb->F + f) * pb->P + j;
}

/* ------------------------------------------------------------------------ */
/* IC precompute (Sec. 3.5): J, r0, W_0 and H = J^T W_0 J in blocks          */
/* ------------------------------------------------------------------------ */
void or_ic_precompute(const or_problem* pb, const double* poses0, const double* depths0,
                      or_ic_pre* pre)
{
    int F = pb->F, N = pb->N, P = pb->P;
    memset(pre->Hff, 0, sizeof(double) * 36 * F);
    memset(pre->Hfd, 0, sizeof(double) * 6 * (size_t)N * F);
    memset(pre->Hdd, 0, sizeof(double) * N);
    for (int n = 0; n < N; ++n) {
        for (int f = 1; f < F; ++f) {
            for (int j = 0; j < P; ++j) {
                size_t id = rid(pb, n, f, j);
                double* J = pre->J + 7 * id;
                pre->valid0[id] = 0;
                pre->r0[id] = 0.0;
                pre->w0[id] = 0.0;
                for (int k = 0; k < 7; ++k) J[k] = 0.0;
                if (!pb->vis[(size_t)n * F + f]) continue;
                double r0;
                int valid = or_ic_residual(pb, poses0, depths0, n, f, j, J, &r0);
                if (!valid) {
                    for (int k = 0; k < 7; ++k) J[k] = 0.0;
                    continue;
                }
                double w0 = or_huber_weight(r0, pb->huber_k);
                pre->valid0[id] = 1;
                pre->r0[id] = r0;
                pre->w0[id] = w0;
                double* Hff = pre->Hff + 36 * f;
                double* Hfd = pre->Hfd + 6 * ((size_t)n * F + f);
                for (int a = 0; a < 6; ++a) {
                    for (int b = 0; b < 6; ++b) Hff[6 * a + b] += w0 * (J[a] * J[b]);
                    Hfd[a] += w0 * J[a] * J[6];
                }
                pre->Hdd[n] += w0 * J[6] * J[6];
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Schur-complement solve of H dp = -g (Sec. 3.5 step 3)                      */
/* ------------------------------------------------------------------------ */
static int cholesky_inplace(double* A, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0.0)) return OR_ERR_NOT_PD;
        double Ljj = sqrt(s);
        A[(size_t)j * n + j] = Ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / Ljj;
        }
    }
    return OR_OK;
}

static void cholesky_solve(const double* L, int n, double* b)
{
    for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * b[k];
        b[i] = s / L[(size_t)i * n + i];
    }
}

/* Solve [Hpp Hpd; Hdp Hdd] [dtheta; dd] = -[g_theta; g_d] with Hpp block
 * diagonal (one 6x6 per target frame) and Hdd diagonal (one scalar per point):
 *   S = Hpp - Hpd Hdd^-1 Hdp,  S dtheta = -(g_theta - Hpd Hdd^-1 g_d),
 *   dd = -Hdd^-1 (g_d + Hdp dtheta).
 * t_anchor: F*3 translations used for the scale gauge.
 * damping = 0 (Gauss-Newton, Sec. 3.5): the scale-gauge prior mu that^T on
 *   the first active frame's translation block makes S definite.
 * damping = lambda > 0 (Levenberg-Marquardt, an option beyond the paper):
 *   every diagonal entry of Hpp and Hdd is multiplied by 1 + lambda, which
 *   makes S definite without the prior; the gauge is then fixed by moving
 *   dtheta along the scale null vector (Delta t_f -= alpha t_f on the active
 *   frames, alpha = t_a . Delta t_a / |t_a|^2 of the anchor frame a) before
 *   the depth back-substitution.
 * S_out (nullable): the (6(F-1))^2 matrix that was factorised. */
int or_schur_solve(int F, int N, const double* Hff, const double* Hfd, const double* Hdd,
                   const double* g_theta, const double* g_d, const double* t_anchor, double damping,
                   double* dtheta, double* dd, double* S_out)
{
    int Fp = F - 1, n6 = 6 * Fp;
    const double ld = 1.0 + damping;
    double* S = (double*)calloc((size_t)n6 * n6, sizeof(double));
    double* b = (double*)calloc(n6, sizeof(double));
    int* active = (int*)calloc(F, sizeof(int));
    for (int f = 1; f < F; ++f) {
        double tr = 0.0;
        for (int a = 0; a < 6; ++a) tr += Hff[36 * f + 7 * a];
        active[f] = tr > 0.0;
        for (int a = 0; a < 6; ++a) {
            for (int c = 0; c < 6; ++c)
                S[(size_t)(6 * (f - 1) + a) * n6 + 6 * (f - 1) + c] =
                    Hff[36 * f + 6 * a + c] * (a == c ? ld : 1.0);
            b[6 * (f - 1) + a] = -g_theta[6 * f + a];
        }
    }
    for (int n = 0; n < N; ++n) {
        if (!(Hdd[n] > 0.0)) continue;
        const double hd = Hdd[n] * ld;
        for (int f = 1; f < F; ++f) {
            const double* hf = Hfd + 6 * ((size_t)n * F + f);
            for (int a = 0; a < 6; ++a) b[6 * (f - 1) + a] += hf[a] * g_d[n] / hd;
            for (int g = 1; g < F; ++g) {
                const double* hg = Hfd + 6 * ((size_t)n * F + g);
                for (int a = 0; a < 6; ++a)
                    for (int c = 0; c < 6; ++c)
                        S[(size_t)(6 * (f - 1) + a) * n6 + 6 * (g - 1) + c] -= hf[a] * hg[c] / hd;
            }
        }
    }
    double mu = 0.0;
    int n_act = 0, anchor = -1;
    for (int f = 1; f < F; ++f) {
        if (!active[f]) continue;
        if (anchor < 0) anchor = f;
        for (int a = 0; a < 6; ++a) mu += S[(size_t)(6 * (f - 1) + a) * n6 + 6 * (f - 1) + a];
        n_act += 6;
    }
    if (n_act > 0) mu /= n_act;
    for (int f = 1; f < F; ++f) {
        if (active[f]) continue;
        for (int a = 0; a < 6; ++a) {
            for (int c = 0; c < n6; ++c) {
                S[(size_t)(6 * (f - 1) + a) * n6 + c] = 0.0;
                S[(size_t)c * n6 + 6 * (f - 1) + a] = 0.0;
            }
            S[(size_t)(6 * (f - 1) + a) * n6 + 6 * (f - 1) + a] = 1.0;
            b[6 * (f - 1) + a] = 0.0;
        }
    }
    if (anchor > 0 && damping == 0.0) {
        const double* ta = t_anchor + 3 * anchor;
        double nt = sqrt(ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2]);
        if (nt > 0.0) {
            double th[3] = {ta[0] / nt, ta[1] / nt, ta[2] / nt};
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c)
                    S[(size_t)(6 * (anchor - 1) + a) * n6 + 6 * (anchor - 1) + c] += mu * th[a] * th[c];
        }
    }
    if (S_out) memcpy(S_out, S, sizeof(double) * n6 * n6);
    int st = cholesky_inplace(S, n6);
    if (st == OR_OK) {
        cholesky_solve(S, n6, b);
        memset(dtheta, 0, sizeof(double) * 6 * F);
        for (int f = 1; f < F; ++f)
            for (int a = 0; a < 6; ++a) dtheta[6 * f + a] = b[6 * (f - 1) + a];
        if (damping > 0.0 && anchor > 0) {
            const double* ta = t_anchor + 3 * anchor;
            const double* da = dtheta + 6 * anchor;
            const double n2 = ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2];
            const double alpha = n2 > 0.0 ? (ta[0] * da[0] + ta[1] * da[1] + ta[2] * da[2]) / n2 : 0.0;
            for (int f = 1; f < F; ++f)
                if (active[f])
                    for (int a = 0; a < 3; ++a) dtheta[6 * f + a] -= alpha * t_anchor[3 * f + a];
        }
        for (int n = 0; n < N; ++n) {
            if (!(Hdd[n] > 0.0)) { dd[n] = 0.0; continue; }
            double s = g_d[n];
            for (int f = 1; f < F; ++f) {
                const double* hf = Hfd + 6 * ((size_t)n * F + f);
                for (int a = 0; a < 6; ++a) s += hf[a] * dtheta[6 * f + a];
            }
            dd[n] = -s / (Hdd[n] * ld);
        }
    }
    free(S);
    free(b);
    free(active);
    return st;
}

/* ------------------------------------------------------------------------ */
/* statistics                                                                */
/* ------------------------------------------------------------------------ */
/* stats[0] Huber energy, [1] RMS residual, [2] valid residual count,
 * [3] max pattern-centre reprojection displacement (px) of the step,
 * [4] |dtheta|_2, [5] |dd|_2 */
enum { ST_ENERGY = 0, ST_RMS, ST_COUNT, ST_MAXDISP, ST_DTHETA, ST_DD, ST_N = 8 };

/* Convergence measure of Sec. 4.1: largest displacement of the reprojected
 * point centres between two parameter sets, over visible (n,f). */
double or_max_reproj_disp(const or_problem* pb, const double* poses_a, const double* depths_a,
                          const double* poses_b, const double* depths_b)
{
    double m = 0.0;
    for (int n = 0; n < pb->N; ++n) {
        double x = (pb->uv[2 * n] - pb->cx) / pb->fx, y = (pb->uv[2 * n + 1] - pb->cy) / pb->fy;
        for (int f = 1; f < pb->F; ++f) {
            if (!pb->vis[(size_t)n * pb->F + f]) continue;
            double wa[2], wb[2];
            or_warp(poses_a + 12 * f, poses_a + 12 * f + 9, depths_a[n], x, y, wa, NULL);
            or_warp(poses_b + 12 * f, poses_b + 12 * f + 9, depths_b[n], x, y, wb, NULL);
            double du = pb->fx * (wa[0] - wb[0]), dv = pb->fy * (wa[1] - wb[1]);
            double dist = sqrt(du * du + dv * dv);
            if (dist > m) m = dist;
        }
    }
    return m;
}

/* ------------------------------------------------------------------------ */
/* IC iteration (Sec. 3.5 steps 1-4, Sec. 3.6 update)                         */
/* ------------------------------------------------------------------------ */
/* Steps 1-2 at the current p: Huber weights from the current residuals and
 * g = J^T W r. Energy/RMS/count over residuals valid now. */
void or_ic_gradient(const or_problem* pb, const or_ic_pre* pre, const double* poses,
                    const double* depths, double* g_theta, double* g_d, double* stats)
{
    int F = pb->F, N = pb->N, P = pb->P;
    memset(g_theta, 0, sizeof(double) * 6 * F);
    memset(g_d, 0, sizeof(double) * N);
    double energy = 0.0, sq = 0.0, cnt = 0.0;
    for (int n = 0; n < N; ++n) {
        for (int f = 1; f < F; ++f) {
            if (!pb->vis[(size_t)n * F + f]) continue;
            const double* R = poses + 12 * f;
            for (int j = 0; j < P; ++j) {
                double r, u[2], q[3];
                if (!residual_at(pb, n, f, j, R, R + 9, depths[n], &r, u, q)) continue;
                energy += or_huber_rho(r, pb->huber_k);
                sq += r * r;
                cnt += 1.0;
                size_t id = rid(pb, n, f, j);
                if (!pre->valid0[id]) continue;
                double w = or_huber_weight(r, pb->huber_k);
                const double* J = pre->J + 7 * id;
                for (int a = 0; a < 6; ++a) g_theta[6 * f + a] += J[a] * w * r;
                g_d[n] += J[6] * w * r;
            }
        }
    }
    stats[ST_ENERGY] = energy;
    stats[ST_RMS] = cnt > 0 ? sqrt(sq / cnt) : 0.0;
    stats[ST_COUNT] = cnt;
}

/* Step 4 by Sec. 3.6: R <- R R0^T exp(omega)^T R0, t <- t - R R0^T dt,
 * d <- d (d0 - dd)/d0 (R on the right-hand sides is the old R). */
void or_ic_update(int F, int N, const double* poses0, const double* depths0,
                  const double* poses, const double* depths, const double* dtheta,
                  const double* dd, double* poses_out, double* depths_out)
{
    memcpy(poses_out, poses, sizeof(double) * 12 * F);
    for (int f = 1; f < F; ++f) {
        const double* R0 = poses0 + 12 * f;
        const double* R = poses + 12 * f;
        double dR[9], dRt[9], R0t[9], A[9], RR0t[9], Rn[9], tmp[3];
        or_so3_exp(dtheta + 6 * f + 3, dR);
        mat3_transpose(dR, dRt);
        mat3_transpose(R0, R0t);
        mat3_mul(R, R0t, RR0t);
        mat3_mul(RR0t, dRt, A);
        mat3_mul(A, R0, Rn);
        mat3_vec(RR0t, dtheta + 6 * f, tmp);
        memcpy(poses_out + 12 * f, Rn, sizeof Rn);
        for (int i = 0; i < 3; ++i) poses_out[12 * f + 9 + i] = R[9 + i] - tmp[i];
    }
    for (int n = 0; n < N; ++n) depths_out[n] = depths[n] * (depths0[n] - dd[n]) / depths0[n];
}

/* Affine brightness (an option beyond the paper; its Sec. 2 notes that
 * direct methods must model lighting): with the residuals of the parameters
 * (poses, depths) and the current (alpha_f, beta_f), each target frame's
 * pair is set so that the warped samples v take the template's weighted
 * mean and spread over the frame's valid residuals (w the Huber weights of
 * those residuals):
 *   alpha = sqrt(var_w(I_0) / var_w(v)),  beta = mean_w(I_0) - alpha mean_w(v).
 * (A least-squares fit of I_0 on v would shrink alpha wherever the
 * geometry is still off, down to alpha ~ 0 that ignores the target image;
 * matching the spreads does not depend on the alignment.) A frame with no
 * residuals or without spread keeps its pair. No-op when the model is off. */
void or_photo_update(const or_problem* pb, const double* poses, const double* depths)
{
    if (!pb->photo) return;
    int F = pb->F, N = pb->N, P = pb->P;
    for (int f = 1; f < F; ++f) {
        const double* R = poses + 12 * f;
        const double* t = R + 9;
        double Sw = 0.0, Sv = 0.0, Svv = 0.0, S0 = 0.0, S00 = 0.0;
        for (int n = 0; n < N; ++n) {
            if (!pb->vis[(size_t)n * F + f]) continue;
            for (int j = 0; j < P; ++j) {
                double r, u[2], q[3];
                if (!residual_at(pb, n, f, j, R, t, depths[n], &r, u, q)) continue;
                const double w = or_huber_weight(r, pb->huber_k);
                int px, py;
                double x, y, v;
                pattern_pixel(pb, n, j, &px, &py, &x, &y);
                const double I0 = pix(frame_img(pb, 0), pb->W, px, py);
                or_bilinear(frame_img(pb, f), pb->W, pb->H, u[0], u[1], &v);  /* the raw sample */
                Sw += w;
                Sv += w * v;
                Svv += w * v * v;
                S0 += w * I0;
                S00 += w * I0 * I0;
            }
        }
        if (!(Sw > 0.0)) continue;
        const double mv = Sv / Sw, m0 = S0 / Sw;
        const double vv = Svv / Sw - mv * mv, v0 = S00 / Sw - m0 * m0;
        if (!(vv > 1e-12) || !(v0 > 1e-12)) continue;
        const double alpha = sqrt(v0 / vv);
        pb->photo[2 * f] = alpha;
        pb->photo[2 * f + 1] = m0 - alpha * mv;
    }
}

/* One IC iteration: steps 1-4. Returns 0 or OR_ERR_NOT_PD. */
int or_ic_step(const or_problem* pb, const or_ic_pre* pre, const double* poses0,
               const double* depths0, const double* poses, const double* depths,
               double* dtheta, double* dd, double* poses_out, double* depths_out,
               double* stats)
{
    int F = pb->F, N = pb->N;
    double* g_theta = (double*)malloc(sizeof(double) * 6 * F);
    double* g_d = (double*)malloc(sizeof(double) * N);
    double* t_anchor = (double*)malloc(sizeof(double) * 3 * F);
    or_ic_gradient(pb, pre, poses, depths, g_theta, g_d, stats);
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < 3; ++i) t_anchor[3 * f + i] = poses0[12 * f + 9 + i];
    int st = or_schur_solve(F, N, pre->Hff, pre->Hfd, pre->Hdd, g_theta, g_d, t_anchor, pb->damping,
                            dtheta, dd, NULL);
    if (st == OR_OK) {
        or_ic_update(F, N, poses0, depths0, poses, depths, dtheta, dd, poses_out, depths_out);
        stats[ST_MAXDISP] = or_max_reproj_disp(pb, poses, depths, poses_out, depths_out);
        /* the brightness pairs from this iteration's residuals (at p_k) */
        or_photo_update(pb, poses, depths);
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 6 * F; ++i) a += dtheta[i] * dtheta[i];
        for (int n = 0; n < N; ++n) b += dd[n] * dd[n];
        stats[ST_DTHETA] = sqrt(a);
        stats[ST_DD] = sqrt(b);
    }
    free(g_theta);
    free(g_d);
    free(t_anchor);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Affine brightness as Gauss-Newton unknowns (IC; an option beyond the      */
/* paper, whose Sec. 2 notes that direct methods must model lighting)        */
/* ------------------------------------------------------------------------ */
/* Each target frame f carries (alpha_f, beta_f) with r = I_0 - (alpha_f I_f +
 * beta_f). In the inverse compositional form the increment acts on the
 * template, as it does for the pose (Sec. 3.5): the template intensities
 * become (1 + da_f) I_0 + db_f, so to first order
 *     r(Delta) = r + J_theta Delta theta_f + J_d Delta d_n + I_0 da_f + db_f,
 * and the two new Jacobian columns, I_0(x) and 1, do not depend on the
 * parameters: H stays fixed at p_0 like the rest of the IC system. The frame
 * blocks become 8 x 8 ([Delta t, omega, da, db]), H_fd 8-vectors. After the
 * solve, (1 + da) I_0 + db = alpha I_f + beta is solved for I_0, which
 * composes the increment into the pair:
 *     alpha' = alpha / (1 + da),  beta' = (beta - db) / (1 + da). */
void or_photo_compose(const double* ab, const double* dab, double* out)
{
    const double s = 1.0 + dab[0];
    out[0] = ab[0] / s;
    out[1] = (ab[1] - dab[1]) / s;
}

/* Schur-complement solve with nb unknowns per frame block (nb = 8: the pose
 * and the brightness pair), otherwise as or_schur_solve: S = Hpp - Hpd
 * Hdd^-1 Hdp, frames without residuals get an identity block, the scale
 * prior mu that that^T (mu = mean diagonal over the pose rows of the active
 * frames) goes on the translation rows of the first active frame (damping =
 * 0), damping scales every diagonal entry of Hpp and Hdd by 1 + lambda and
 * then moves the translations along the scale null vector. Hff: F*nb*nb,
 * Hfd: N*F*nb, g_theta: F*nb; dtheta: F*nb out. */
static int schur_solve_nb(int nb, int F, int N, const double* Hff, const double* Hfd, const double* Hdd,
                          const double* g_theta, const double* g_d, const double* t_anchor, double damping,
                          double* dtheta, double* dd)
{
    int Fp = F - 1, n = nb * Fp;
    const double ld = 1.0 + damping;
    double* S = (double*)calloc((size_t)n * n, sizeof(double));
    double* b = (double*)calloc(n, sizeof(double));
    int* active = (int*)calloc(F, sizeof(int));
    for (int f = 1; f < F; ++f) {
        double tr = 0.0;
        for (int a = 0; a < 6; ++a) tr += Hff[((size_t)f * nb + a) * nb + a];
        active[f] = tr > 0.0;
        for (int a = 0; a < nb; ++a) {
            for (int c = 0; c < nb; ++c)
                S[(size_t)(nb * (f - 1) + a) * n + nb * (f - 1) + c] =
                    Hff[((size_t)f * nb + a) * nb + c] * (a == c ? ld : 1.0);
            b[nb * (f - 1) + a] = -g_theta[nb * f + a];
        }
    }
    for (int p = 0; p < N; ++p) {
        if (!(Hdd[p] > 0.0)) continue;
        const double hd = Hdd[p] * ld;
        for (int f = 1; f < F; ++f) {
            const double* hf = Hfd + nb * ((size_t)p * F + f);
            for (int a = 0; a < nb; ++a) b[nb * (f - 1) + a] += hf[a] * g_d[p] / hd;
            for (int g = 1; g < F; ++g) {
                const double* hg = Hfd + nb * ((size_t)p * F + g);
                for (int a = 0; a < nb; ++a)
                    for (int c = 0; c < nb; ++c)
                        S[(size_t)(nb * (f - 1) + a) * n + nb * (g - 1) + c] -= hf[a] * hg[c] / hd;
            }
        }
    }
    double mu = 0.0;
    int n_act = 0, anchor = -1;
    for (int f = 1; f < F; ++f) {
        if (!active[f]) continue;
        if (anchor < 0) anchor = f;
        for (int a = 0; a < 6; ++a) mu += S[(size_t)(nb * (f - 1) + a) * n + nb * (f - 1) + a];
        n_act += 6;
    }
    if (n_act > 0) mu /= n_act;
    for (int f = 1; f < F; ++f) {
        if (active[f]) continue;
        for (int a = 0; a < nb; ++a) {
            for (int c = 0; c < n; ++c) {
                S[(size_t)(nb * (f - 1) + a) * n + c] = 0.0;
                S[(size_t)c * n + nb * (f - 1) + a] = 0.0;
            }
            S[(size_t)(nb * (f - 1) + a) * n + nb * (f - 1) + a] = 1.0;
            b[nb * (f - 1) + a] = 0.0;
        }
    }
    if (anchor > 0 && damping == 0.0) {
        const double* ta = t_anchor + 3 * anchor;
        double nt = sqrt(ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2]);
        if (nt > 0.0) {
            double th[3] = {ta[0] / nt, ta[1] / nt, ta[2] / nt};
            for (int a = 0; a < 3; ++a)
                for (int c = 0; c < 3; ++c)
                    S[(size_t)(nb * (anchor - 1) + a) * n + nb * (anchor - 1) + c] += mu * th[a] * th[c];
        }
    }
    int st = cholesky_inplace(S, n);
    if (st == OR_OK) {
        cholesky_solve(S, n, b);
        memset(dtheta, 0, sizeof(double) * nb * F);
        for (int f = 1; f < F; ++f)
            for (int a = 0; a < nb; ++a) dtheta[nb * f + a] = b[nb * (f - 1) + a];
        if (damping > 0.0 && anchor > 0) {
            const double* ta = t_anchor + 3 * anchor;
            const double* da = dtheta + nb * anchor;
            const double n2 = ta[0] * ta[0] + ta[1] * ta[1] + ta[2] * ta[2];
            const double alpha = n2 > 0.0 ? (ta[0] * da[0] + ta[1] * da[1] + ta[2] * da[2]) / n2 : 0.0;
            for (int f = 1; f < F; ++f)
                if (active[f])
                    for (int a = 0; a < 3; ++a) dtheta[nb * f + a] -= alpha * t_anchor[3 * f + a];
        }
        for (int p = 0; p < N; ++p) {
            if (!(Hdd[p] > 0.0)) { dd[p] = 0.0; continue; }
            double s = g_d[p];
            for (int f = 1; f < F; ++f) {
                const double* hf = Hfd + nb * ((size_t)p * F + f);
                for (int a = 0; a < nb; ++a) s += hf[a] * dtheta[nb * f + a];
            }
            dd[p] = -s / (Hdd[p] * ld);
        }
    }
    free(S);
    free(b);
    free(active);
    return st;
}

/* One IC iteration with the brightness pairs pb->photo as unknowns (steps
 * 1-4 of Sec. 3.5 over the 8-parameter frame blocks; the pose and depth
 * updates of Sec. 3.6; the pairs by or_photo_compose). H comes from the
 * precompute's rows and W_0 (valid at p_0), extended by the columns I_0 and
 * 1; g = J^T W r over the residuals valid now and at p_0, with the weights
 * of the current residuals; with pb->photo_prior > 0 a prior pulls the pairs
 * toward (1, 0). dtheta: F*6, dab: F*2 (frame 0: zero). */
int or_ic_step_joint(const or_problem* pb, const or_ic_pre* pre, const double* poses0,
                     const double* depths0, const double* poses, const double* depths,
                     double* dtheta, double* dab, double* dd, double* poses_out, double* depths_out,
                     double* stats)
{
    int F = pb->F, N = pb->N, P = pb->P;
    if (!pb->photo || F < 2) return OR_ERR_NOT_PD;
    double* Hff = (double*)calloc((size_t)64 * F, sizeof(double));
    double* Hfd = (double*)calloc((size_t)8 * N * F, sizeof(double));
    double* g8 = (double*)calloc((size_t)8 * F, sizeof(double));
    double* g_d = (double*)calloc(N, sizeof(double));
    double* d8 = (double*)calloc((size_t)8 * F, sizeof(double));
    double* t_anchor = (double*)malloc(sizeof(double) * 3 * F);
    double energy = 0.0, sq = 0.0, cnt = 0.0;
    for (int n = 0; n < N; ++n) {
        for (int f = 1; f < F; ++f) {
            if (!pb->vis[(size_t)n * F + f]) continue;
            const double* R = poses + 12 * f;
            for (int j = 0; j < P; ++j) {
                size_t id = rid(pb, n, f, j);
                int px, py;
                double x, y;
                pattern_pixel(pb, n, j, &px, &py, &x, &y);
                /* the frame-block row [J_theta, I_0, 1] and the depth column */
                double Jf[8];
                const double* J = pre->J + 7 * id;
                for (int a = 0; a < 6; ++a) Jf[a] = J[a];
                Jf[6] = pix(frame_img(pb, 0), pb->W, px, py);
                Jf[7] = 1.0;
                if (pre->valid0[id]) {
                    const double w0 = pre->w0[id];
                    double* hff = Hff + 64 * f;
                    double* hfd = Hfd + 8 * ((size_t)n * F + f);
                    for (int a = 0; a < 8; ++a) {
                        for (int b = 0; b < 8; ++b) hff[8 * a + b] += w0 * (Jf[a] * Jf[b]);
                        hfd[a] += w0 * Jf[a] * J[6];
                    }
                }
                double r, u[2], q[3];
                if (!residual_at(pb, n, f, j, R, R + 9, depths[n], &r, u, q)) continue;
                energy += or_huber_rho(r, pb->huber_k);
                sq += r * r;
                cnt += 1.0;
                if (!pre->valid0[id]) continue;
                const double w = or_huber_weight(r, pb->huber_k);
                for (int a = 0; a < 8; ++a) g8[8 * f + a] += Jf[a] * w * r;
                g_d[n] += J[6] * w * r;
            }
        }
    }
    stats[ST_ENERGY] = energy;
    stats[ST_RMS] = cnt > 0 ? sqrt(sq / cnt) : 0.0;
    stats[ST_COUNT] = cnt;
    /* prior on the pairs: lambda W_f ((ln alpha_f)^2 + beta_f^2) / 2 with W_f =
     * sum w0 of the frame (its H_bb); to first order in the increment ln
     * alpha' = ln alpha - da and beta' = beta - db, i.e. residuals (ln alpha,
     * beta) with Jacobian -I on (da, db): H += W I, g -= W (ln alpha, beta) */
    if (pb->photo_prior > 0.0)
        for (int f = 1; f < F; ++f) {
            const double w = pb->photo_prior * Hff[64 * f + 63];
            Hff[64 * f + 54] += w;
            Hff[64 * f + 63] += w;
            g8[8 * f + 6] -= w * log(pb->photo[2 * f]);
            g8[8 * f + 7] -= w * pb->photo[2 * f + 1];
        }
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < 3; ++i) t_anchor[3 * f + i] = poses0[12 * f + 9 + i];
    int st = schur_solve_nb(8, F, N, Hff, Hfd, pre->Hdd, g8, g_d, t_anchor, pb->damping, d8, dd);
    if (st == OR_OK) {
        for (int f = 0; f < F; ++f) {
            for (int a = 0; a < 6; ++a) dtheta[6 * f + a] = d8[8 * f + a];
            dab[2 * f] = d8[8 * f + 6];
            dab[2 * f + 1] = d8[8 * f + 7];
        }
        or_ic_update(F, N, poses0, depths0, poses, depths, dtheta, dd, poses_out, depths_out);
        stats[ST_MAXDISP] = or_max_reproj_disp(pb, poses, depths, poses_out, depths_out);
        for (int f = 1; f < F; ++f) {
            double ab[2];
            or_photo_compose(pb->photo + 2 * f, dab + 2 * f, ab);
            pb->photo[2 * f] = ab[0];
            pb->photo[2 * f + 1] = ab[1];
        }
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 6 * F; ++i) a += dtheta[i] * dtheta[i];
        for (int n = 0; n < N; ++n) b += dd[n] * dd[n];
        stats[ST_DTHETA] = sqrt(a);
        stats[ST_DD] = sqrt(b);
    }
    free(Hff);
    free(Hfd);
    free(g8);
    free(g_d);
    free(d8);
    free(t_anchor);
    return st;
}

/* ------------------------------------------------------------------------ */
/* FC iteration (the plain method: Jacobians and Hessian every iteration)    */
/* ------------------------------------------------------------------------ */
void or_fc_linearize(const or_problem* pb, const double* poses, const double* depths,
                     double* Hff, double* Hfd, double* Hdd, double* g_theta, double* g_d,
                     double* stats)
{
    int F = pb->F, N = pb->N, P = pb->P;
    memset(Hff, 0, sizeof(double) * 36 * F);
    memset(Hfd, 0, sizeof(double) * 6 * (size_t)N * F);
    memset(Hdd, 0, sizeof(double) * N);
    memset(g_theta, 0, sizeof(double) * 6 * F);
    memset(g_d, 0, sizeof(double) * N);
    double energy = 0.0, sq = 0.0, cnt = 0.0;
    for (int n = 0; n < N; ++n) {
        for (int f = 1; f < F; ++f) {
            if (!pb->vis[(size_t)n * F + f]) continue;
            for (int j = 0; j < P; ++j) {
                double J[7], r;
                if (!or_fc_residual(pb, poses, depths, n, f, j, J, &r)) continue;
                double w = or_huber_weight(r, pb->huber_k);
                energy += or_huber_rho(r, pb->huber_k);
                sq += r * r;
                cnt += 1.0;
                double* hff = Hff + 36 * f;
                double* hfd = Hfd + 6 * ((size_t)n * F + f);
                for (int a = 0; a < 6; ++a) {
                    for (int b = 0; b < 6; ++b) hff[6 * a + b] += w * (J[a] * J[b]);
                    hfd[a] += w * J[a] * J[6];
                    g_theta[6 * f + a] += w * J[a] * r;
                }
                Hdd[n] += w * J[6] * J[6];
                g_d[n] += w * J[6] * r;
            }
        }
    }
    stats[ST_ENERGY] = energy;
    stats[ST_RMS] = cnt > 0 ? sqrt(sq / cnt) : 0.0;
    stats[ST_COUNT] = cnt;
}

/* Boxplus (Sec. 3 Notation): T <- exp([upsilon, omega]) T, d <- d + dd. */
void or_fc_update(int F, int N, const double* poses, const double* depths, const double* dtheta,
                  const double* dd, double* poses_out, double* depths_out)
{
    memcpy(poses_out, poses, sizeof(double) * 12 * F);
    for (int f = 1; f < F; ++f) {
        double dR[9], dt[3], Rn[9], tn[3];
        or_se3_exp(dtheta + 6 * f, dR, dt);
        mat3_mul(dR, poses + 12 * f, Rn);
        mat3_vec(dR, poses + 12 * f + 9, tn);
        memcpy(poses_out + 12 * f, Rn, sizeof Rn);
        for (int i = 0; i < 3; ++i) poses_out[12 * f + 9 + i] = tn[i] + dt[i];
    }
    for (int n = 0; n < N; ++n) depths_out[n] = depths[n] + dd[n];
}

int or_fc_step(const or_problem* pb, const double* poses, const double* depths, double* dtheta,
               double* dd, double* poses_out, double* depths_out, double* stats)
{
    int F = pb->F, N = pb->N;
    double* Hff = (double*)malloc(sizeof(double) * 36 * F);
    double* Hfd = (double*)malloc(sizeof(double) * 6 * (size_t)N * F);
    double* Hdd = (double*)malloc(sizeof(double) * N);
    double* g_theta = (double*)malloc(sizeof(double) * 6 * F);
    double* g_d = (double*)malloc(sizeof(double) * N);
    double* t_anchor = (double*)malloc(sizeof(double) * 3 * F);
    or_fc_linearize(pb, poses, depths, Hff, Hfd, Hdd, g_theta, g_d, stats);
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < 3; ++i) t_anchor[3 * f + i] = poses[12 * f + 9 + i];
    int st = or_schur_solve(F, N, Hff, Hfd, Hdd, g_theta, g_d, t_anchor, pb->damping, dtheta, dd, NULL);
    if (st == OR_OK) {
        or_fc_update(F, N, poses, depths, dtheta, dd, poses_out, depths_out);
        stats[ST_MAXDISP] = or_max_reproj_disp(pb, poses, depths, poses_out, depths_out);
        or_photo_update(pb, poses, depths);
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 6 * F; ++i) a += dtheta[i] * dtheta[i];
        for (int n = 0; n < N; ++n) b += dd[n] * dd[n];
        stats[ST_DTHETA] = sqrt(a);
        stats[ST_DD] = sqrt(b);
    }
    free(Hff);
    free(Hfd);
    free(Hdd);
    free(g_theta);
    free(g_d);
    free(t_anchor);
    return st;
}

/* FC with the brightness pairs as unknowns (an option beyond the paper): the
 * residual r = I_0 - (alpha_f v + beta_f), v = I_f(W(x; p)), is linearised at
 * the current parameters in all of them, so the frame block's two new
 * columns are dr/dalpha = -v and dr/dbeta = -1 and the pairs are updated
 * additively. Jrow (9): [dr/d(upsilon, omega) (6), -v, -1, dr/dd]. */
int or_fc_residual_joint(const or_problem* pb, const double* poses, const double* depths, int n, int f,
                         int j, double* Jrow, double* r)
{
    double J7[7], u[2], q[3], v = 0.0;
    const double* R = poses + 12 * f;
    for (int k = 0; k < 9; ++k) Jrow[k] = 0.0;
    if (!or_fc_residual(pb, poses, depths, n, f, j, J7, r)) return 0;
    residual_at(pb, n, f, j, R, R + 9, depths[n], r, u, q);
    or_bilinear(frame_img(pb, f), pb->W, pb->H, u[0], u[1], &v);
    for (int k = 0; k < 6; ++k) Jrow[k] = J7[k];
    Jrow[6] = -v;
    Jrow[7] = -1.0;
    Jrow[8] = J7[6];
    return 1;
}

/* One FC iteration with the pairs pb->photo as unknowns: H = J^T W J and
 * g = J^T W r over the 8-parameter frame blocks at the current parameters,
 * the 8 (F - 1) Schur solve (or_schur_solve's gauge and damping), the
 * boxplus pose update, d <- d + dd and (alpha, beta) += (da, db). dtheta:
 * F*6, dab: F*2. (No prior: or_ic_step_joint's prior belongs to the IC
 * form.) */
int or_fc_step_joint(const or_problem* pb, const double* poses, const double* depths, double* dtheta,
                     double* dab, double* dd, double* poses_out, double* depths_out, double* stats)
{
    int F = pb->F, N = pb->N, P = pb->P;
    if (!pb->photo || F < 2) return OR_ERR_NOT_PD;
    double* Hff = (double*)calloc((size_t)64 * F, sizeof(double));
    double* Hfd = (double*)calloc((size_t)8 * N * F, sizeof(double));
    double* Hdd = (double*)calloc(N, sizeof(double));
    double* g8 = (double*)calloc((size_t)8 * F, sizeof(double));
    double* g_d = (double*)calloc(N, sizeof(double));
    double* d8 = (double*)calloc((size_t)8 * F, sizeof(double));
    double* t_anchor = (double*)malloc(sizeof(double) * 3 * F);
    double energy = 0.0, sq = 0.0, cnt = 0.0;
    for (int n = 0; n < N; ++n) {
        for (int f = 1; f < F; ++f) {
            if (!pb->vis[(size_t)n * F + f]) continue;
            for (int j = 0; j < P; ++j) {
                double J[9], r;
                if (!or_fc_residual_joint(pb, poses, depths, n, f, j, J, &r)) continue;
                const double w = or_huber_weight(r, pb->huber_k);
                energy += or_huber_rho(r, pb->huber_k);
                sq += r * r;
                cnt += 1.0;
                double* hff = Hff + 64 * f;
                double* hfd = Hfd + 8 * ((size_t)n * F + f);
                for (int a = 0; a < 8; ++a) {
                    for (int b = 0; b < 8; ++b) hff[8 * a + b] += w * (J[a] * J[b]);
                    hfd[a] += w * J[a] * J[8];
                    g8[8 * f + a] += w * J[a] * r;
                }
                Hdd[n] += w * J[8] * J[8];
                g_d[n] += w * J[8] * r;
            }
        }
    }
    stats[ST_ENERGY] = energy;
    stats[ST_RMS] = cnt > 0 ? sqrt(sq / cnt) : 0.0;
    stats[ST_COUNT] = cnt;
    for (int f = 0; f < F; ++f)
        for (int i = 0; i < 3; ++i) t_anchor[3 * f + i] = poses[12 * f + 9 + i];
    int st = schur_solve_nb(8, F, N, Hff, Hfd, Hdd, g8, g_d, t_anchor, pb->damping, d8, dd);
    if (st == OR_OK) {
        for (int f = 0; f < F; ++f) {
            for (int a = 0; a < 6; ++a) dtheta[6 * f + a] = d8[8 * f + a];
            dab[2 * f] = d8[8 * f + 6];
            dab[2 * f + 1] = d8[8 * f + 7];
        }
        or_fc_update(F, N, poses, depths, dtheta, dd, poses_out, depths_out);
        stats[ST_MAXDISP] = or_max_reproj_disp(pb, poses, depths, poses_out, depths_out);
        for (int f = 1; f < F; ++f) {
            pb->photo[2 * f] += dab[2 * f];
            pb->photo[2 * f + 1] += dab[2 * f + 1];
        }
        double a = 0.0, b = 0.0;
        for (int i = 0; i < 6 * F; ++i) a += dtheta[i] * dtheta[i];
        for (int n = 0; n < N; ++n) b += dd[n] * dd[n];
        stats[ST_DTHETA] = sqrt(a);
        stats[ST_DD] = sqrt(b);
    }
    free(Hff);
    free(Hfd);
    free(Hdd);
    free(g8);
    free(g_d);
    free(d8);
    free(t_anchor);
    return st;
}

/* Residual statistics only (energy, RMS, count) at a parameter set. */
void or_eval(const or_problem* pb, const double* poses, const double* depths, double* stats)
{
    double energy = 0.0, sq = 0.0, cnt = 0.0;
    for (int n = 0; n < pb->N; ++n)
        for (int f = 1; f < pb->F; ++f) {
            if (!pb->vis[(size_t)n * pb->F + f]) continue;
            const double* R = poses + 12 * f;
            for (int j = 0; j < pb->P; ++j) {
                double r, u[2], q[3];
                if (!residual_at(pb, n, f, j, R, R + 9, depths[n], &r, u, q)) continue;
                energy += or_huber_rho(r, pb->huber_k);
                sq += r * r;
                cnt += 1.0;
            }
        }
    stats[ST_ENERGY] = energy;
    stats[ST_RMS] = cnt > 0 ? sqrt(sq / cnt) : 0.0;
    stats[ST_COUNT] = cnt;
}
