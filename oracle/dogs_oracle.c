/*
 * dogs_oracle.c -- plain, slow FP64 CPU oracle for the DOGS hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it follows:
 *   - Gaussian primitive and covariance factorisation Sigma = R S S^T R^T
 *     (Sec. 3.1, Eq. 1 and the text under it);
 *   - alpha blending C = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)
 *     (Sec. 3.1, Eq. 2) with the usual tile rasteriser rules: EWA projection
 *     J W Sigma W^T J^T + 0.3 I, degree<=3 real SH colour, alpha clamped to
 *     0.99, pairs with alpha < 1/255 skipped, stop before T drops below 1e-4;
 *   - the analytic adjoint of all of the above;
 *   - the block ADMM updates: x-step penalty rho/2 ||x - z + u||^2 (Eq. 7,
 *     Eq. 8a, per-property form Eq. 12a), consensus z = mean over the blocks
 *     holding a Gaussian of (x + u) (Eq. 8b in its complete form, Appendix
 *     "Proof of Eq. 8b"), dual update u += x - z (Eq. 8c, Eq. 12c),
 *     over-relaxation (Sec. 3.3) and the residuals of Eq. 9.
 *
 * Layout (its own): one Gaussian = P = 11 + 3K doubles
 *   [mu(3), q(4) = (w,x,y,z), log-scale(3), SH f (K x 3, coefficient-major),
 *    opacity logit(1)],  K = (D+1)^2 SH coefficients for degree D.
 * A projected record = 16 doubles
 *   [mx, my, a, b, c, opacity, r, g, b, depth, raw_r, raw_g, raw_b,
 *    radius, tiles, visible].
 *
 * Parity status: every function here is pinned by the CPU tests (closed
 * forms, brute force, finite differences, hand-worked ADMM examples).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OC_PI 3.14159265358979323846

/* Host threads for the per-Gaussian and per-pixel loops (OpenMP when built  */
/* with it).  The default is one: results are then bit-for-bit reproducible; */
/* with more threads only the order of the FP64 additions into a record's    */
/* gradient changes.  The CPU baseline of the benchmark times both.           */
static int g_threads = 1;
void oc_set_threads(int n) { g_threads = n > 0 ? n : 1; }
int oc_get_threads(void) { return g_threads; }
int oc_have_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy;
    double R[9];      /* world -> camera rotation, row-major */
    double t[3];      /* world -> camera translation          */
    double campos[3]; /* camera centre in world coordinates   */
    double near_z;
} oc_cam;

enum { REC_MX = 0, REC_MY, REC_A, REC_B, REC_C, REC_OP, REC_R, REC_G, REC_BL, REC_DEPTH,
       REC_RAWR, REC_RAWG, REC_RAWB, REC_RADIUS, REC_TILES, REC_VIS, REC_N };

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                       */
/* ------------------------------------------------------------------------ */
static void matmul(const double* A, const double* B, double* C, int n, int k, int m)
{   /* C (n x m) = A (n x k) B (k x m) */
    for (int i = 0; i < n; i++)
        for (int j = 0; j < m; j++) {
            double s = 0.0;
            for (int l = 0; l < k; l++) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}
static void transpose(const double* A, double* At, int n, int m)
{   /* At (m x n) = A^T, A is n x m */
    for (int i = 0; i < n; i++)
        for (int j = 0; j < m; j++) At[j * n + i] = A[i * m + j];
}

/* ------------------------------------------------------------------------ */
/* real spherical harmonics, from the definition                             */
/* Y_l0 = K_l0 P_l(z);  m>0: (-1)^m sqrt2 K_lm P_l^(m)(z) Re((x+iy)^m);      */
/* m<0: (-1)^|m| sqrt2 K_l|m| P_l^(|m|)(z) Im((x+iy)^|m|), where P_l^(m) is  */
/* the m-th derivative of the Legendre polynomial P_l and                    */
/* K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  This is the real basis with    */
/* the Condon-Shortley phase, evaluated on the unit sphere.                  */
/* ------------------------------------------------------------------------ */
static double fact(int n) { double f = 1.0; for (int i = 2; i <= n; i++) f *= i; return f; }
static double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

/* coefficients c[j] of z^j of the m-th derivative of P_l, j = 0..l */
static void legendre_deriv_coef(int l, int m, double* c)
{
    double p[8] = {0};
    for (int k = 0; 2 * k <= l; k++)
        p[l - 2 * k] = ldexp(1.0, -l) * ((k & 1) ? -1.0 : 1.0) * binom(l, k) * binom(2 * l - 2 * k, l);
    for (int d = 0; d < m; d++) {
        for (int j = 0; j < l; j++) p[j] = p[j + 1] * (j + 1);
        p[l] = 0.0;
    }
    for (int j = 0; j <= l; j++) c[j] = p[j];
}
static double poly_eval(const double* c, int deg, double z)
{
    double s = 0.0, zp = 1.0;
    for (int j = 0; j <= deg; j++) { s += c[j] * zp; zp *= z; }
    return s;
}
static double poly_deriv_eval(const double* c, int deg, double z)
{
    double s = 0.0, zp = 1.0;
    for (int j = 1; j <= deg; j++) { s += j * c[j] * zp; zp *= z; }
    return s;
}
/* Re and Im of (x + i y)^m */
static void cplx_pow(double x, double y, int m, double* re, double* im)
{
    double a = 1.0, b = 0.0;
    for (int i = 0; i < m; i++) { double na = a * x - b * y, nb = a * y + b * x; a = na; b = nb; }
    *re = a; *im = b;
}

/* value and gradient (w.r.t. the three components, the z-polynomial taken as */
/* written) of Y_lm at direction d.  grad may be NULL.                         */
double oc_sh_basis(int l, int m, const double* d, double* grad)
{
    int am = m < 0 ? -m : m;
    double c[8];
    legendre_deriv_coef(l, am, c);
    double K = sqrt((2.0 * l + 1.0) / (4.0 * OC_PI) * fact(l - am) / fact(l + am));
    double Q = poly_eval(c, l, d[2]), dQ = poly_deriv_eval(c, l, d[2]);
    if (m == 0) {
        if (grad) { grad[0] = 0.0; grad[1] = 0.0; grad[2] = K * dQ; }
        return K * Q;
    }
    double s = ((am & 1) ? -1.0 : 1.0) * sqrt(2.0) * K;
    double re, im, re1, im1;
    cplx_pow(d[0], d[1], am, &re, &im);
    cplx_pow(d[0], d[1], am - 1, &re1, &im1);
    if (m > 0) {
        if (grad) { grad[0] = s * Q * am * re1; grad[1] = -s * Q * am * im1; grad[2] = s * dQ * re; }
        return s * Q * re;
    }
    if (grad) { grad[0] = s * Q * am * im1; grad[1] = s * Q * am * re1; grad[2] = s * dQ * im; }
    return s * Q * im;
}

/* k = l*l + l + m  ->  (l, m) */
static void sh_lm(int k, int* l, int* m)
{
    int L = 0;
    while ((L + 1) * (L + 1) <= k) L++;
    *l = L; *m = k - L * L - L;
}

/* ------------------------------------------------------------------------ */
/* rotation from a unit quaternion (w, x, y, z) and its partial derivatives  */
/* ------------------------------------------------------------------------ */
static void quat_to_rot(const double* q, double* R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
/* dR[k] = dR/dq_k for k = w, x, y, z */
static void quat_to_rot_partials(const double* q, double dR[4][9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double Dw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
    double Dx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    double Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
    double Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
    memcpy(dR[0], Dw, sizeof Dw); memcpy(dR[1], Dx, sizeof Dx);
    memcpy(dR[2], Dy, sizeof Dy); memcpy(dR[3], Dz, sizeof Dz);
}

/* ------------------------------------------------------------------------ */
/* forward projection of one Gaussian into one view                          */
/* ------------------------------------------------------------------------ */
typedef struct {
    double t[3], qn[4], qnorm, Rq[9], s[3], M[9], Sigma[9], J[6], T[6], Sp[4], det;
    double d[3], vnorm, o;
} proj_tmp;

static double frac_dist(double v) { return fabs(v - floor(v + 0.5)); }
static int iclamp(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* camera-frame point, each row summed in a fixed order */
static void to_camera(const oc_cam* cam, const double* mu, double* t)
{
    for (int i = 0; i < 3; i++) {
        double s = cam->R[3 * i + 0] * mu[0];
        s = s + cam->R[3 * i + 1] * mu[1];
        s = s + cam->R[3 * i + 2] * mu[2];
        t[i] = s + cam->t[i];
    }
}

/* ------------------------------------------------------------------------ */
/* tile culling at binning: a reading of Eq. 2's 1/255 rule                   */
/* ------------------------------------------------------------------------ */
/* A pixel at offset d from the mean can only be composited if               */
/* o exp(-q(d) / 2) >= 1/255, q(d) = a dx^2 + 2 b dx dy + c dy^2, i.e.        */
/* q(d) <= 2 ln(255 o).  A tile of the record's rectangle is binned only if   */
/* the minimum of q over the box of its pixel centres is within that bound,  */
/* widened to tau = 2 ln(255 o) (1 + 2^-10) + 2^-6 so that no FP32 decision   */
/* of the compositing can fall outside it.  Dropped pairs would all be       */
/* skipped by the compositing, so images and gradients are unchanged.        */
static double cull_tau(double o) { return 2.0 * log(255.0 * o) * (1.0 + 1.0 / 1024.0) + 1.0 / 64.0; }

static double dclamp(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* minimum of the convex q over [X0, X1] x [Y0, Y1] (offsets from the mean):  */
/* 0 if the box holds the mean, else the least of the four edge minima, each */
/* edge minimiser being the unconstrained one clamped to the edge.           */
static double box_qmin(double a, double b, double c, double X0, double X1, double Y0, double Y1)
{
    if (X0 <= 0.0 && 0.0 <= X1 && Y0 <= 0.0 && 0.0 <= Y1) return 0.0;
    double best = INFINITY, xs[2] = {X0, X1}, ys[2] = {Y0, Y1};
    for (int i = 0; i < 2; i++) {
        double X = xs[i], y = dclamp(-b * X / c, Y0, Y1);
        best = fmin(best, a * X * X + 2.0 * b * X * y + c * y * y);
        double Y = ys[i], x = dclamp(-b * Y / a, X0, X1);
        best = fmin(best, a * x * x + 2.0 * b * x * Y + c * Y * Y);
    }
    return best;
}

/* exported for the tests: box_qmin */
double oc_box_qmin(double a, double b, double c, double X0, double X1, double Y0, double Y1)
{
    return box_qmin(a, b, c, X0, X1, Y0, Y1);
}

/* q-minimum of tile (tx, ty) for a record; the box spans the pixel centres */
static double tile_qmin(const double* rec, int tx, int ty, int tile_w, int tile_h)
{
    double X0 = tx * tile_w + 0.5 - rec[REC_MX], X1 = tx * tile_w + tile_w - 0.5 - rec[REC_MX];
    double Y0 = ty * tile_h + 0.5 - rec[REC_MY], Y1 = ty * tile_h + tile_h - 0.5 - rec[REC_MY];
    return box_qmin(rec[REC_A], rec[REC_B], rec[REC_C], X0, X1, Y0, Y1);
}

static int project_one(const double* x, int K, const oc_cam* cam, int tile_w, int tile_h,
                       double* rec, int32_t* rect, float* depth_key, double* margin, proj_tmp* tp)
{
    proj_tmp tmp; proj_tmp* T = tp ? tp : &tmp;
    for (int i = 0; i < REC_N; i++) rec[i] = 0.0;
    rect[0] = rect[1] = rect[2] = rect[3] = 0;
    *depth_key = 0.0f;
    double mg = INFINITY;
    const double* mu = x;
    to_camera(cam, mu, T->t);
    double tx = T->t[0], ty = T->t[1], tz = T->t[2];
    mg = fmin(mg, fabs(tz - cam->near_z) / fabs(cam->near_z));
    if (!(tz > cam->near_z)) { *margin = mg; return 0; }
    double xn = tx / tz, yn = ty / tz;
    double limx = 1.3 * 0.5 * cam->width / cam->fx, limy = 1.3 * 0.5 * cam->height / cam->fy;
    mg = fmin(mg, fabs(fabs(xn) - limx) / limx);
    mg = fmin(mg, fabs(fabs(yn) - limy) / limy);
    if (fabs(xn) > limx || fabs(yn) > limy) { *margin = mg; return 0; }
    /* Sigma = R S S^T R^T */
    const double* q = x + 3;
    T->qnorm = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; i++) T->qn[i] = q[i] / T->qnorm;
    quat_to_rot(T->qn, T->Rq);
    for (int j = 0; j < 3; j++) T->s[j] = exp(x[7 + j]);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) T->M[3 * i + j] = T->Rq[3 * i + j] * T->s[j];
    double Mt[9];
    transpose(T->M, Mt, 3, 3);
    matmul(T->M, Mt, T->Sigma, 3, 3, 3);
    /* EWA: J = d(pixel)/d(camera point), T = J W, Sigma' = T Sigma T^T + 0.3 I */
    double J[6] = {cam->fx / tz, 0.0, -cam->fx * tx / (tz * tz),
                   0.0, cam->fy / tz, -cam->fy * ty / (tz * tz)};
    memcpy(T->J, J, sizeof J);
    matmul(J, cam->R, T->T, 2, 3, 3);
    double TS[6], Tt[6];
    matmul(T->T, T->Sigma, TS, 2, 3, 3);
    transpose(T->T, Tt, 2, 3);
    matmul(TS, Tt, T->Sp, 2, 3, 2);
    T->Sp[0] += 0.3; T->Sp[3] += 0.3;
    T->det = T->Sp[0] * T->Sp[3] - T->Sp[1] * T->Sp[2];
    if (!(T->det > 0.0)) { *margin = mg; return 0; }
    double a = T->Sp[3] / T->det, b = -T->Sp[1] / T->det, c = T->Sp[0] / T->det;
    double mid = 0.5 * (T->Sp[0] + T->Sp[3]);
    double lmax = mid + sqrt(fmax(mid * mid - T->det, 0.0));
    double r3 = 3.0 * sqrt(lmax);
    int radius = (int)ceil(r3);
    mg = fmin(mg, frac_dist(r3));
    double mx = cam->fx * xn + cam->cx, my = cam->fy * yn + cam->cy;
    int TX = (cam->width + tile_w - 1) / tile_w, TY = (cam->height + tile_h - 1) / tile_h;
    double ex0 = (mx - radius) / tile_w, ex1 = (mx + radius) / tile_w;
    double ey0 = (my - radius) / tile_h, ey1 = (my + radius) / tile_h;
    mg = fmin(mg, fmin(fmin(frac_dist(ex0), frac_dist(ex1)), fmin(frac_dist(ey0), frac_dist(ey1))));
    int x0 = iclamp((int)floor(ex0), 0, TX), x1 = iclamp((int)floor(ex1) + 1, 0, TX);
    int y0 = iclamp((int)floor(ey0), 0, TY), y1 = iclamp((int)floor(ey1) + 1, 0, TY);
    int tiles = (x1 - x0) * (y1 - y0);
    *margin = mg;
    if (tiles <= 0) return 0;
    /* colour: sum_k f_k Y_k(d) + 0.5, clamped at 0 */
    double v[3] = {mu[0] - cam->campos[0], mu[1] - cam->campos[1], mu[2] - cam->campos[2]};
    T->vnorm = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int i = 0; i < 3; i++) T->d[i] = v[i] / T->vnorm;
    double raw[3] = {0.5, 0.5, 0.5};
    for (int k = 0; k < K; k++) {
        int l, m; sh_lm(k, &l, &m);
        double Y = oc_sh_basis(l, m, T->d, NULL);
        for (int ch = 0; ch < 3; ch++) raw[ch] += x[10 + 3 * k + ch] * Y;
    }
    for (int ch = 0; ch < 3; ch++) mg = fmin(mg, fabs(raw[ch]));   /* colour clamp decision */
    *margin = mg;
    T->o = 1.0 / (1.0 + exp(-x[10 + 3 * K]));
    rec[REC_MX] = mx; rec[REC_MY] = my;
    rec[REC_A] = a; rec[REC_B] = b; rec[REC_C] = c;
    rec[REC_OP] = T->o;
    for (int ch = 0; ch < 3; ch++) { rec[REC_RAWR + ch] = raw[ch]; rec[REC_R + ch] = raw[ch] > 0 ? raw[ch] : 0.0; }
    rec[REC_DEPTH] = tz;
    rec[REC_RADIUS] = radius; rec[REC_TILES] = tiles; rec[REC_VIS] = 1.0;
    rect[0] = x0; rect[1] = y0; rect[2] = x1; rect[3] = y1;
    *depth_key = (float)tz;
    /* margin of every tile-culling decision */
    double tau = cull_tau(T->o);
    for (int ty = y0; ty < y1; ty++)
        for (int tx = x0; tx < x1; tx++)
            mg = fmin(mg, fabs(tile_qmin(rec, tx, ty, tile_w, tile_h) - tau) / (1.0 + fabs(tau)));
    *margin = mg;
    return 1;
}

/* Project n Gaussians (params n x P) into one view.  Returns #visible.      */
int oc_project(int n, int sh_degree, const double* params, const oc_cam* cam,
               int tile_w, int tile_h, double* rec, int32_t* rect, float* depth_key,
               double* margin)
{
    int K = (sh_degree + 1) * (sh_degree + 1), P = 11 + 3 * K, vis = 0;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1024) reduction(+ : vis)
    for (int i = 0; i < n; i++)
        vis += project_one(params + (int64_t)i * P, K, cam, tile_w, tile_h, rec + (int64_t)i * REC_N,
                           rect + 4 * (int64_t)i, depth_key + i, margin + i, NULL);
    return vis;
}

/* ------------------------------------------------------------------------ */
/* binning: one (key, value) per covered tile, key = (tile << 32) | bits     */
/* of the float depth, sorted ascending by (key, value)                      */
/* ------------------------------------------------------------------------ */
typedef struct { uint64_t key; uint32_t val; } kv;
static int kv_cmp(const void* A, const void* B)
{
    const kv* a = (const kv*)A; const kv* b = (const kv*)B;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->val != b->val) return a->val < b->val ? -1 : 1;
    return 0;
}

/* Records r of all views: view[r], rect[4r..], depth_key[r], visible[r],    */
/* rec[REC_N r..].  Per view: tile_off[v], tiles_x[v].  Writes keys/vals      */
/* (count returned; at most `capacity` written) and ranges[2*tile] for        */
/* n_tiles tiles.  cull != 0 drops the tiles the record cannot reach (above). */
static int keep_tile(int cull, const double* rec, int tx, int ty, int tile_w, int tile_h)
{
    return !cull || tile_qmin(rec, tx, ty, tile_w, tile_h) <= cull_tau(rec[REC_OP]);
}

int64_t oc_bin_sort(int64_t n_rec, const int32_t* view, const int32_t* rect, const float* depth_key,
                    const int32_t* visible, const int32_t* tile_off, const int32_t* tiles_x,
                    int64_t n_tiles, int64_t capacity, uint64_t* keys, uint32_t* vals,
                    uint32_t* ranges, const double* rec, int tile_w, int tile_h, int cull)
{
    int64_t M = 0;
    for (int64_t r = 0; r < n_rec; r++) {
        if (!visible[r]) continue;
        for (int ty = rect[4 * r + 1]; ty < rect[4 * r + 3]; ty++)
            for (int tx = rect[4 * r]; tx < rect[4 * r + 2]; tx++)
                M += keep_tile(cull, rec + r * REC_N, tx, ty, tile_w, tile_h);
    }
    if (M > capacity) return M;
    kv* list = (kv*)malloc(sizeof(kv) * (M > 0 ? M : 1));
    int64_t p = 0;
    for (int64_t r = 0; r < n_rec; r++) {
        if (!visible[r]) continue;
        uint32_t dbits; memcpy(&dbits, &depth_key[r], 4);
        for (int ty = rect[4 * r + 1]; ty < rect[4 * r + 3]; ty++)
            for (int tx = rect[4 * r]; tx < rect[4 * r + 2]; tx++) {
                if (!keep_tile(cull, rec + r * REC_N, tx, ty, tile_w, tile_h)) continue;
                uint64_t tile = (uint64_t)tile_off[view[r]] + (uint64_t)ty * tiles_x[view[r]] + tx;
                list[p].key = (tile << 32) | dbits;
                list[p].val = (uint32_t)r;
                p++;
            }
    }
    qsort(list, M, sizeof(kv), kv_cmp);
    for (int64_t i = 0; i < M; i++) { keys[i] = list[i].key; vals[i] = list[i].val; }
    /* range of tile t = [first index with tile >= t, first index with tile >= t+1) */
    int64_t j = 0;
    for (int64_t t = 0; t < n_tiles; t++) {
        while (j < M && (int64_t)(list[j].key >> 32) < t) j++;
        int64_t s = j;
        while (j < M && (int64_t)(list[j].key >> 32) == t) j++;
        ranges[2 * t] = (uint32_t)s; ranges[2 * t + 1] = (uint32_t)j;
    }
    free(list);
    return M;
}

/* ------------------------------------------------------------------------ */
/* per-pixel front-to-back compositing (Eq. 2)                               */
/* ------------------------------------------------------------------------ */
#define ALPHA_MAX 0.99
#define ALPHA_MIN (1.0 / 255.0)
#define T_MIN 1e-4

typedef struct { uint32_t rec; double alpha, alpha_raw, G, T, dx, dy; } pair_t;

/* composites one pixel; fills `pairs` (if non-NULL) with composited pairs    */
/* margin: relative distance of the value decisions (1/255 skip, T stop) from */
/* their thresholds; margin_grad (may be NULL): of the 0.99 clamp, which only   */
/* decides gradients                                                           */
static int composite_pixel_seen(int px, int py, const uint32_t* vals, uint32_t beg, uint32_t end,
                                const double* rec, const double* bg, double* C, double* Tout,
                                uint32_t* last, double* margin, double* margin_grad, pair_t* pairs,
                                uint32_t* seen)
{
    double T = 1.0, col[3] = {0, 0, 0}, mg = INFINITY, mg2 = INFINITY;
    int np = 0;
    uint32_t lst = 0;
    if (seen) *seen = end - beg;                 /* no stop: every position examined */
    for (uint32_t j = beg; j < end; j++) {
        const double* g = rec + (int64_t)vals[j] * REC_N;
        double dx = g[REC_MX] - (px + 0.5), dy = g[REC_MY] - (py + 0.5);
        double power = -0.5 * (g[REC_A] * dx * dx + g[REC_C] * dy * dy) - g[REC_B] * dx * dy;
        if (power > 0.0) power = 0.0;   /* positive-definite conic: only rounding makes it positive */
        double G = exp(power);
        double ar = g[REC_OP] * G;
        double alpha = ar < ALPHA_MAX ? ar : ALPHA_MAX;
        mg = fmin(mg, fabs(alpha - ALPHA_MIN) / ALPHA_MIN);
        if (alpha < ALPHA_MIN) continue;
        mg2 = fmin(mg2, fabs(ar - ALPHA_MAX) / ALPHA_MAX);   /* clamp decides the gradient */
        double Tn = T * (1.0 - alpha);
        mg = fmin(mg, fabs(Tn - T_MIN) / T_MIN);
        if (Tn < T_MIN) {
            if (seen) *seen = j - beg + 1;
            break;
        }
        for (int ch = 0; ch < 3; ch++) col[ch] += g[REC_R + ch] * alpha * T;
        if (pairs) {
            pairs[np].rec = vals[j]; pairs[np].alpha = alpha; pairs[np].alpha_raw = ar;
            pairs[np].G = G; pairs[np].T = T; pairs[np].dx = dx; pairs[np].dy = dy;
        }
        np++;
        T = Tn;
        lst = j - beg + 1;
    }
    for (int ch = 0; ch < 3; ch++) C[ch] = col[ch] + T * bg[ch];
    *Tout = T; *last = lst; *margin = mg;
    if (margin_grad) *margin_grad = mg2;
    return np;
}

static int composite_pixel(int px, int py, const uint32_t* vals, uint32_t beg, uint32_t end,
                           const double* rec, const double* bg, double* C, double* Tout,
                           uint32_t* last, double* margin, double* margin_grad, pair_t* pairs)
{
    return composite_pixel_seen(px, py, vals, beg, end, rec, bg, C, Tout, last, margin, margin_grad, pairs,
                                NULL);
}

/* Work counts of the compositing per pixel: seen = list positions examined  */
/* (up to and including the one that stops the pixel), used = Eq. 2 terms     */
/* composited (alpha >= 1/255, before the stop).                              */
void oc_rasterize_counts(int width, int height, int tile_w, int tile_h, int64_t tile_off,
                         const uint32_t* vals, const uint32_t* ranges, const double* rec,
                         uint32_t* seen, uint32_t* used)
{
    const double bg[3] = {0, 0, 0};
    int TX = (width + tile_w - 1) / tile_w;
    for (int py = 0; py < height; py++)
        for (int px = 0; px < width; px++) {
            int64_t tile = tile_off + (int64_t)(py / tile_h) * TX + px / tile_w;
            int64_t p = (int64_t)py * width + px;
            double C[3], Tf, mg;
            uint32_t lst;
            used[p] = (uint32_t)composite_pixel_seen(px, py, vals, ranges[2 * tile], ranges[2 * tile + 1], rec,
                                                     bg, C, &Tf, &lst, &mg, NULL, NULL, &seen[p]);
        }
}

/* Render one view of size W x H whose tiles are numbered from tile_off.      */
/* image is 3 x H x W (planar).                                              */
void oc_rasterize_fwd(int width, int height, int tile_w, int tile_h, int64_t tile_off,
                      const uint32_t* vals, const uint32_t* ranges, const double* rec,
                      const double* bg, double* image, double* T_final, uint32_t* last,
                      double* margin, double* margin_grad)
{
    int TX = (width + tile_w - 1) / tile_w;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 4)
    for (int py = 0; py < height; py++)
        for (int px = 0; px < width; px++) {
            int64_t tile = tile_off + (int64_t)(py / tile_h) * TX + px / tile_w;
            double C[3];
            int64_t p = (int64_t)py * width + px;
            composite_pixel(px, py, vals, ranges[2 * tile], ranges[2 * tile + 1], rec, bg, C,
                            &T_final[p], &last[p], &margin[p], &margin_grad[p], NULL);
            for (int ch = 0; ch < 3; ch++) image[(int64_t)ch * width * height + p] = C[ch];
        }
}

/* Adjoint of the compositing: accumulates dL/d(record) into drec (n_rec x 9: */
/* dmx, dmy, da, db, dc, dopacity, dr, dg, db).                               */
void oc_rasterize_bwd(int width, int height, int tile_w, int tile_h, int64_t tile_off,
                      const uint32_t* vals, const uint32_t* ranges, const double* rec,
                      const double* bg, const double* dL_dimage, double* drec)
{
    int TX = (width + tile_w - 1) / tile_w;
    int64_t maxlen = 0;
    for (int64_t t = tile_off; t < tile_off + (int64_t)TX * ((height + tile_h - 1) / tile_h); t++)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
#pragma omp parallel num_threads(g_threads)
    {
    pair_t* pairs = (pair_t*)malloc(sizeof(pair_t) * (maxlen > 0 ? maxlen : 1));
    double* S = (double*)malloc(sizeof(double) * 3 * (maxlen + 1));
#pragma omp for schedule(dynamic, 4)
    for (int py = 0; py < height; py++)
        for (int px = 0; px < width; px++) {
            int64_t tile = tile_off + (int64_t)(py / tile_h) * TX + px / tile_w;
            int64_t p = (int64_t)py * width + px;
            double C[3], Tf, mg; uint32_t lst;
            int np = composite_pixel(px, py, vals, ranges[2 * tile], ranges[2 * tile + 1], rec, bg, C,
                                     &Tf, &lst, &mg, NULL, pairs);
            double gpix[3];
            for (int ch = 0; ch < 3; ch++) gpix[ch] = dL_dimage[(int64_t)ch * width * height + p];
            /* S_i = sum_{j > i} c_j alpha_j T_j + T_final * bg (suffix sums) */
            for (int ch = 0; ch < 3; ch++) S[3 * (np - 1 >= 0 ? np - 1 : 0) + ch] = Tf * bg[ch];
            for (int i = np - 2; i >= 0; i--) {
                const double* gn = rec + (int64_t)pairs[i + 1].rec * REC_N;
                for (int ch = 0; ch < 3; ch++)
                    S[3 * i + ch] = S[3 * (i + 1) + ch] + gn[REC_R + ch] * pairs[i + 1].alpha * pairs[i + 1].T;
            }
            for (int i = 0; i < np; i++) {
                const pair_t* pr = &pairs[i];
                const double* g = rec + (int64_t)pr->rec * REC_N;
                double* dg = drec + (int64_t)pr->rec * 9;
                double dalpha = 0.0, d[9];
                for (int ch = 0; ch < 3; ch++) {
                    d[6 + ch] = gpix[ch] * pr->alpha * pr->T;
                    dalpha += gpix[ch] * (g[REC_R + ch] * pr->T - S[3 * i + ch] / (1.0 - pr->alpha));
                }
                int nd = 6;
                if (pr->alpha_raw < ALPHA_MAX) {                /* clamp active: no gradient */
                    d[5] = dalpha * pr->G;
                    double dpower = dalpha * g[REC_OP] * pr->G;
                    double dx = pr->dx, dy = pr->dy;
                    d[0] = dpower * (-(g[REC_A] * dx + g[REC_B] * dy));
                    d[1] = dpower * (-(g[REC_C] * dy + g[REC_B] * dx));
                    d[2] = dpower * (-0.5 * dx * dx);
                    d[3] = dpower * (-dx * dy);
                    d[4] = dpower * (-0.5 * dy * dy);
                    nd = 0;
                }
                for (int j = nd; j < 9; j++) {
#pragma omp atomic
                    dg[j] += d[j];
                }
            }
        }
    free(pairs); free(S);
    }
}

/* ------------------------------------------------------------------------ */
/* adjoint of the projection: dL/d(record) -> dL/d(params), accumulated      */
/* ------------------------------------------------------------------------ */
static void project_bwd_one(const double* x, int K, const oc_cam* cam, int tile_w, int tile_h,
                            const double* dr, double* dx)
{
    double rec[REC_N], mg; int32_t rect[4]; float dk; proj_tmp T;
    if (!project_one(x, K, cam, tile_w, tile_h, rec, rect, &dk, &mg, &T)) return;
    int P = 11 + 3 * K;
    (void)P;
    double tz = T.t[2], tx = T.t[0], ty = T.t[1];
    /* opacity logit */
    dx[10 + 3 * K] += dr[5] * T.o * (1.0 - T.o);
    /* colour -> SH coefficients and view direction */
    double gcol[3], dd[3] = {0, 0, 0};
    for (int ch = 0; ch < 3; ch++) gcol[ch] = rec[REC_RAWR + ch] > 0 ? dr[6 + ch] : 0.0;
    for (int k = 0; k < K; k++) {
        int l, m; sh_lm(k, &l, &m);
        double gY[3];
        double Y = oc_sh_basis(l, m, T.d, gY);
        for (int ch = 0; ch < 3; ch++) {
            dx[10 + 3 * k + ch] += gcol[ch] * Y;
            for (int i = 0; i < 3; i++) dd[i] += gcol[ch] * x[10 + 3 * k + ch] * gY[i];
        }
    }
    double ddot = dd[0] * T.d[0] + dd[1] * T.d[1] + dd[2] * T.d[2];
    for (int i = 0; i < 3; i++) dx[i] += (dd[i] - T.d[i] * ddot) / T.vnorm;
    /* conic = inverse of Sigma'; gradient w.r.t. the inverse as a symmetric   */
    /* matrix Gi, then dL/dSigma' = -Sinv Gi Sinv                               */
    double Sinv[4] = {rec[REC_A], rec[REC_B], rec[REC_B], rec[REC_C]};
    double Gi[4] = {dr[2], 0.5 * dr[3], 0.5 * dr[3], dr[4]};
    double tmp[4], G[4];
    matmul(Sinv, Gi, tmp, 2, 2, 2);
    matmul(tmp, Sinv, G, 2, 2, 2);
    for (int i = 0; i < 4; i++) G[i] = -G[i];
    /* Sigma' = T Sigma T^T:  dSigma = T^T G T,  dT = 2 G T Sigma */
    double Tt[6], GT[6], dSigma[9], dT[6], GTS[6];
    transpose(T.T, Tt, 2, 3);
    matmul(G, T.T, GT, 2, 2, 3);
    matmul(Tt, GT, dSigma, 3, 2, 3);
    matmul(GT, T.Sigma, GTS, 2, 3, 3);
    for (int i = 0; i < 6; i++) dT[i] = 2.0 * GTS[i];
    /* T = J W:  dJ = dT W^T */
    double Wt[9], dJ[6];
    transpose(cam->R, Wt, 3, 3);
    matmul(dT, Wt, dJ, 2, 3, 3);
    /* J(t) and mean2d(t) -> dt */
    double fx = cam->fx, fy = cam->fy, dt[3] = {0, 0, 0};
    dt[0] += dJ[2] * (-fx / (tz * tz));
    dt[1] += dJ[5] * (-fy / (tz * tz));
    dt[2] += dJ[0] * (-fx / (tz * tz)) + dJ[2] * (2.0 * fx * tx / (tz * tz * tz))
           + dJ[4] * (-fy / (tz * tz)) + dJ[5] * (2.0 * fy * ty / (tz * tz * tz));
    dt[0] += dr[0] * fx / tz;
    dt[1] += dr[1] * fy / tz;
    dt[2] += -dr[0] * fx * tx / (tz * tz) - dr[1] * fy * ty / (tz * tz);
    /* t = W mu + t_w */
    double dmu[3];
    matmul(Wt, dt, dmu, 3, 3, 1);
    for (int i = 0; i < 3; i++) dx[i] += dmu[i];
    /* Sigma = M M^T, M = R S */
    double dM[9];
    double dSs[9];
    for (int i = 0; i < 9; i++) dSs[i] = dSigma[i] + dSigma[(i % 3) * 3 + i / 3];
    matmul(dSs, T.M, dM, 3, 3, 3);
    double dR[9];
    for (int j = 0; j < 3; j++) {
        double ds = 0.0;
        for (int i = 0; i < 3; i++) { ds += dM[3 * i + j] * T.Rq[3 * i + j]; dR[3 * i + j] = dM[3 * i + j] * T.s[j]; }
        dx[7 + j] += ds * T.s[j];
    }
    double P4[4][9], dqn[4];
    quat_to_rot_partials(T.qn, P4);
    for (int k = 0; k < 4; k++) {
        dqn[k] = 0.0;
        for (int i = 0; i < 9; i++) dqn[k] += dR[i] * P4[k][i];
    }
    double qd = 0.0;
    for (int k = 0; k < 4; k++) qd += dqn[k] * T.qn[k];
    for (int k = 0; k < 4; k++) dx[3 + k] += (dqn[k] - T.qn[k] * qd) / T.qnorm;
}

/* drec: n x 9 for this view's records; dparams: n x P, accumulated.         */
void oc_project_bwd(int n, int sh_degree, const double* params, const oc_cam* cam,
                    int tile_w, int tile_h, const double* drec, double* dparams)
{
    int K = (sh_degree + 1) * (sh_degree + 1), P = 11 + 3 * K;
#pragma omp parallel for num_threads(g_threads) schedule(dynamic, 1024)
    for (int i = 0; i < n; i++)
        project_bwd_one(params + (int64_t)i * P, K, cam, tile_w, tile_h, drec + (int64_t)i * 9,
                        dparams + (int64_t)i * P);
}

/* ------------------------------------------------------------------------ */
/* ADMM                                                                      */
/* ------------------------------------------------------------------------ */
/* property group of parameter index j: 0 mean, 1 rotation, 2 scale,          */
/* 3 SH features, 4 opacity (the paper's order p, q, s, f, o)                 */
static int group_of(int j, int K)
{
    if (j < 3) return 0;
    if (j < 7) return 1;
    if (j < 10) return 2;
    if (j < 10 + 3 * K) return 3;
    return 4;
}
/* learning-rate slot: the five groups with SH split into DC and the rest     */
static int lr_slot(int j, int K)
{
    int g = group_of(j, K);
    if (g < 3) return g;
    if (g == 3) return j < 13 ? 3 : 4;
    return 5;
}

/* One Adam step on f_k + sum_grp rho_grp/2 ||x - z + u||^2 for every local  */
/* copy (Eq. 8a / 12a); the penalty applies to shared copies only.          */
void oc_adam_admm_step(int64_t n_copies, int sh_degree, double* x, const double* grad,
                       double* m, double* v, const double* z, const double* u,
                       const int32_t* copy_gid, const uint8_t* shared, const double* rho,
                       const double* lr, double b1, double b2, double eps, int step)
{
    int K = (sh_degree + 1) * (sh_degree + 1), P = 11 + 3 * K;
    double c1 = 1.0 - pow(b1, step), c2 = 1.0 - pow(b2, step);
    for (int64_t c = 0; c < n_copies; c++)
        for (int j = 0; j < P; j++) {
            int64_t e = c * P + j;
            double g = grad[e];
            if (shared[c]) g += rho[group_of(j, K)] * (x[e] - z[(int64_t)copy_gid[c] * P + j] + u[e]);
            m[e] = b1 * m[e] + (1.0 - b1) * g;
            v[e] = b2 * v[e] + (1.0 - b2) * g * g;
            double mh = m[e] / c1, vh = v[e] / c2;
            x[e] -= lr[lr_slot(j, K)] * mh / (sqrt(vh) + eps);
        }
}

/* Consensus over globals (CSR g_off / g_copies).  On entry z holds z^t, on   */
/* exit z^{t+1}.  Shared globals (two or more copies):                        */
/*   xh_k = alpha x_k + (1 - alpha) z^t        (over-relaxation, Sec. 3.3)    */
/*   z    = (1/n_i) sum_k (xh_k + u_k)         (Eq. 8b, complete form)        */
/*   u_k += xh_k - z                           (Eq. 8c)                       */
/* Unshared globals: z = x, u untouched.  res (may be NULL) gets, per group,  */
/* the squared primal residual sum ||x_k - z||^2 in res[0..4] and the squared */
/* dual residual rho^2 n_i ||z^{t+1} - z^t||^2 in res[5..9] (Eq. 9), shared   */
/* globals only.                                                              */
void oc_consensus(int64_t n_glob, int sh_degree, const int64_t* g_off, const int32_t* g_copies,
                  const double* x, double* u, double* z, double alpha, const double* rho,
                  double* res)
{
    int K = (sh_degree + 1) * (sh_degree + 1), P = 11 + 3 * K;
    if (res) for (int i = 0; i < 10; i++) res[i] = 0.0;
    for (int64_t i = 0; i < n_glob; i++) {
        int64_t b = g_off[i], e = g_off[i + 1], n = e - b;
        double* zi = z + i * P;
        if (n == 1) {
            const double* xc = x + (int64_t)g_copies[b] * P;
            for (int j = 0; j < P; j++) zi[j] = xc[j];
            continue;
        }
        for (int j = 0; j < P; j++) {
            double zprev = zi[j], acc = 0.0;
            for (int64_t k = b; k < e; k++) {
                int64_t c = g_copies[k];
                double xh = alpha * x[c * P + j] + (1.0 - alpha) * zprev;
                acc += xh + u[c * P + j];
            }
            double znew = acc / (double)n;
            for (int64_t k = b; k < e; k++) {
                int64_t c = g_copies[k];
                double xh = alpha * x[c * P + j] + (1.0 - alpha) * zprev;
                u[c * P + j] += xh - znew;
                if (res) res[group_of(j, K)] += (x[c * P + j] - znew) * (x[c * P + j] - znew);
            }
            if (res) {
                double r = rho[group_of(j, K)];
                res[5 + group_of(j, K)] += r * r * (double)n * (znew - zprev) * (znew - zprev);
            }
            zi[j] = znew;
        }
    }
}
