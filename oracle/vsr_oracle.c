/*
 * vsr_oracle.c -- plain FP64 CPU oracle of the visual-sphere rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The product (the CUDA
 * library and its Python binding) never calls it, includes it or shares code
 * with it.
 *
 * Everything here is computed in double precision, by brute force over every
 * (pixel, triangle) pair, in the order the paper states the method:
 *
 *   map      Universal perspective 2D->3D transform (Sec. 2 "Universal
 *            perspective", eq. of the 2D->3D transformation) with the
 *            parameter limits (Sec. "Universal perspective parameters and
 *            limits") and the view-coordinate normalisation of the AOV remark
 *            (Sec. 2, remark on AOV types).  The global delta (Sec. 1.1.1,
 *            "Global delta") is the reciprocal of the largest per-component
 *            fwidth of the map.
 *   setup    edge-plane normals ||A x B||, ||B x C||, ||C x A|| (Sec. 1.1),
 *            the miter / smallest-circle vector S (Sec. 1.1.2), the hard
 *            normal N and plane offset d = A.N (Sec. 1.1.4, depth equation).
 *   raster   the four plane distances of the rasterization equation
 *            (Sec. 1.1.2, eq. "rasterization"), gpstep / gbpxstep (Sec. 1.1.1),
 *            bstep for the centre test, ray-plane depth r = (A.N)/(G.N), and
 *            the front-to-back mask merge of Sec. 1.4 (hidden surface
 *            occlusion).
 *   shade    the same merge applied to a shade pass c_t |N-hat . G| (the
 *            differentiable workload's image, Sec. 1.4 and Sec. 1.1.4).
 *   gradient the analytic adjoint of that image (and of coverage and depth)
 *            through the merge, gpstep / min, the plane distances, the
 *            set-up and the map; the map's lens tangents by complex step.
 *            Pinned by central differences of the functions above.
 *
 * The only shortcut is that the miter-plane test of gbpxstep is evaluated
 * before the three edge-plane tests: a pair that fails it is not a fragment
 * by definition, so skipping the remaining arithmetic changes no result.
 *
 * Readings where the paper is silent or inconsistent (each one is listed
 * with its reason in the design notes of the repository):
 *   R1  R = sqrt(x^2 + l*y^2) as in the equation (the listing squares l).
 *   R3  pixel centres f = ((i+1/2)/W, (j+1/2)/H), aspect a = W/H.
 *   R5  s is clamped to [0.5, 1] unless strict limits ask for [0.8, 1].
 *   R6  pixels where asin is undefined are invalid: map (0,0,0,0).
 *   R7  R = 0 uses the limit of sin(theta)/R.
 *   R8  fwidth = |central difference along i| + |along j| of the map
 *       function at the neighbouring pixel centres, one-sided next to an
 *       invalid neighbour, 0 when both are invalid.
 *   R10 two-sided triangles: sigma = sign(A'.(B' x C')) orients all normals.
 *   R11 ties g == 0 in the centre test count as inside iff the first
 *       nonzero component of the edge normal is positive; each edge's cross
 *       product is taken with its vertices in a canonical order (bit pattern
 *       of the world-space FP32 coordinates) so shared edges get exactly
 *       opposite normals.
 *   R15 front-to-back order = ascending (r, t); id/depth from the nearest
 *       centre-inside fragment; fragments with r <= 0 or non-finite r are
 *       dropped.
 *   R17 the miter plane's distance G.S-hat - |S| is divided by sin(rho),
 *       rho the cap's angular radius, before the global-delta step.  The
 *       edge distances G.n are sines of angular distances (unit slope at the
 *       edge) but the miter distance has slope sin(rho) at its rim; the
 *       per-fragment pstep of the paper's listing divides by fwidth(g),
 *       which removes any such scale, and the global delta stands in for
 *       that denominator only for unit-slope distances.  Without the factor
 *       the miter ramp is 1/sin(rho) pixels wide and a small triangle never
 *       reaches full coverage.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_PI 3.14159265358979323846

/* Record layout of one set-up triangle (doubles). */
enum {
    REC_N1 = 0,  /* edge normal of A,B (3) */
    REC_N2 = 3,  /* edge normal of B,C (3) */
    REC_N3 = 6,  /* edge normal of C,A (3) */
    REC_S = 9,   /* miter unit vector S-hat (3) */
    REC_C = 12,  /* |S| = cosine of the cap radius rho */
    REC_N = 13,  /* hard normal N (3) */
    REC_D = 16,  /* A'.N */
    REC_VALID = 17,
    REC_SIGMA = 18,
    REC_SR = 19, /* sin(rho) = sqrt(1 - |S|^2) */
    ORC_REC = 20
};

int orc_record_size(void) { return ORC_REC; }

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------
 * Parameter limits (Sec. "Universal perspective parameters and limits").
 * k in [-1,1], l in [0,1], s in [0.8,1] (strict) or [0.5,1] (reading R5),
 * Omega in degrees clamped to [1, Omega_max] with
 * Omega_max = (k > 0 ? 179 : 180) / max(|k|, 1/2).
 * out = {k, l, s, omega_deg}.
 */
void orc_limits(double k, double l, double s, double omega_deg, int strict, double* out)
{
    k = clampd(k, -1.0, 1.0);
    l = clampd(l, 0.0, 1.0);
    s = clampd(s, strict ? 0.8 : 0.5, 1.0);
    double kmag = fabs(k) > 0.5 ? fabs(k) : 0.5;
    double omax = (k > 0.0 ? 179.0 : 180.0) / kmag;
    omega_deg = clampd(omega_deg, 1.0, omax);
    out[0] = k;
    out[1] = l;
    out[2] = s;
    out[3] = omega_deg;
}

/* ------------------------------------------------------------------------
 * View coordinates from texture coordinates (remark on AOV types, Sec. 2):
 * centred 2f-1, then normalised for the AOV type.
 * aov: 0 horizontal, 1 diagonal, 2 vertical, 3 horizontal 4x3.
 */
void orc_view_coord(double fs, double ft, double aspect, int aov, double* xy)
{
    double x = 2.0 * fs - 1.0, y = 2.0 * ft - 1.0;
    switch (aov) {
    case 1: /* diagonal: [a, 1] / sqrt(1 + a^2) */
        x = x * aspect / sqrt(1.0 + aspect * aspect);
        y = y / sqrt(1.0 + aspect * aspect);
        break;
    case 2: /* vertical: [a, 1] */
        x = x * aspect;
        break;
    case 3: /* horizontal 4x3: [a, 1] / (4/3) */
        x = x * aspect / (4.0 / 3.0);
        y = y / (4.0 / 3.0);
        break;
    default: /* horizontal: [1, 1/a] */
        y = y / aspect;
        break;
    }
    xy[0] = x;
    xy[1] = y;
}

/* ------------------------------------------------------------------------
 * Universal perspective 2D->3D (Sec. "Transformation of 2D->3D"):
 *   R     = sqrt(x^2 + l y^2)                                   (reading R1)
 *   theta = atan(tan(k Omega/2) R)/k   k > 0
 *           Omega/2 R                  k = 0
 *           asin(sin(k Omega/2) R)/k   k < 0
 *   v     = normalize(x sin(theta)/R, y sin(theta)/R / (l(1-s)+s), cos(theta))
 * p = {k, l, s, omega_deg} after limits.  Returns 0 where asin is undefined
 * (reading R6), 1 otherwise.
 */
int orc_map_dir(double x, double y, const double* p, double* v)
{
    double k = p[0], l = p[1], s = p[2];
    double half = p[3] * ORC_PI / 360.0; /* Omega/2 in radians */
    double R = sqrt(x * x + l * y * y);
    double theta, sin_over_R;
    if (k > 0.0) {
        double tk = tan(k * half);
        theta = atan(tk * R) / k;
        sin_over_R = R > 0.0 ? sin(theta) / R : tk / k; /* reading R7 */
    } else if (k == 0.0) {
        theta = half * R;
        sin_over_R = R > 0.0 ? sin(theta) / R : half;
    } else {
        double sk = sin(k * half);
        double arg = sk * R;
        if (arg > 1.0 || arg < -1.0) {
            v[0] = v[1] = v[2] = 0.0;
            return 0;
        }
        theta = asin(arg) / k;
        sin_over_R = R > 0.0 ? sin(theta) / R : sk / k;
    }
    double w[3] = {x * sin_over_R, y * sin_over_R / (l * (1.0 - s) + s), cos(theta)};
    double n = sqrt(dot3(w, w));
    v[0] = w[0] / n;
    v[1] = w[1] / n;
    v[2] = w[2] / n;
    return 1;
}

/* Map direction at a texture coordinate (fs, ft) of a W x H picture. */
static int map_at(double fs, double ft, double aspect, int aov, const double* p, double* v)
{
    double xy[2];
    orc_view_coord(fs, ft, aspect, aov, xy);
    return orc_map_dir(xy[0], xy[1], p, v);
}

/* Vectorised map function at arbitrary texture coordinates (used by the
 * supersampling and area pins).  v: n x 3, valid: n. */
void orc_map_dirs(int64_t n, const double* fs, const double* ft, int W, int H, const double* p, int aov,
                  double* v, int32_t* valid)
{
    double aspect = (double)W / (double)H;
    for (int64_t q = 0; q < n; ++q) valid[q] = map_at(fs[q], ft[q], aspect, aov, p, v + 3 * q);
}

/* ------------------------------------------------------------------------
 * Universal perspective 3D->2D (Sec. "Transformation of 3D->2D"):
 *   theta = acos(v_z / sqrt(v_x^2 + l v_y^2 + v_z^2))
 *   R     = tan(k theta)/tan(k Omega/2)   k > 0
 *           theta/(Omega/2)               k = 0
 *           sin(k theta)/sin(k Omega/2)   k < 0
 *   (x,y) = (v_x, v_y) R / sqrt(v_x^2 + l v_y^2) * (1, l(1-s)+s)
 * Used only as a round-trip pin of the 2D->3D map.
 */
void orc_map_inverse(const double* v, const double* p, double* xy)
{
    double k = p[0], l = p[1], s = p[2];
    double half = p[3] * ORC_PI / 360.0;
    double theta = acos(v[2] / sqrt(v[0] * v[0] + l * v[1] * v[1] + v[2] * v[2]));
    double R;
    if (k > 0.0)
        R = tan(k * theta) / tan(k * half);
    else if (k == 0.0)
        R = theta / half;
    else
        R = sin(k * theta) / sin(k * half);
    double rho = sqrt(v[0] * v[0] + l * v[1] * v[1]);
    if (rho == 0.0) {
        xy[0] = xy[1] = 0.0;
        return;
    }
    xy[0] = v[0] * R / rho;
    xy[1] = v[1] * R / rho * (l * (1.0 - s) + s);
}

/* ------------------------------------------------------------------------
 * Perspective map with global delta (Sec. 1.1.1 "Global delta"):
 *   out[(j*W + i)*4 + 0..2] = v(i, j),  out[...+3] = delta(i, j)
 *   delta = 1 / max_c (|d_i v_c| + |d_j v_c|)           (reading R8)
 * Invalid pixels are (0,0,0,0).  The map function is evaluated on the
 * (W+2) x (H+2) grid of pixel centres including a one-pixel border.
 */
typedef struct {
    int W, H, aov;
    const double* p;
    double* grid; /* (H+2)*(W+2)*3 */
    int* gvalid;
    double* out;
    int next_row;
    int phase;
} map_job;

static void* map_worker(void* arg)
{
    map_job* J = (map_job*)arg;
    const int W = J->W, H = J->H, GW = W + 2;
    const double aspect = (double)W / (double)H;
    for (;;) {
        int row = __atomic_fetch_add(&J->next_row, 1, __ATOMIC_RELAXED);
        if (J->phase == 0) {
            if (row >= H + 2) break;
            int j = row - 1;
            for (int gi = 0; gi < GW; ++gi) {
                int i = gi - 1;
                double* v = J->grid + ((size_t)row * GW + gi) * 3;
                J->gvalid[(size_t)row * GW + gi] =
                    map_at((i + 0.5) / W, (j + 0.5) / H, aspect, J->aov, J->p, v);
            }
        } else {
            if (row >= H) break;
            int j = row;
            for (int i = 0; i < W; ++i) {
                double* o = J->out + ((size_t)j * W + i) * 4;
                size_t c0 = (size_t)(j + 1) * GW + (i + 1);
                if (!J->gvalid[c0]) {
                    o[0] = o[1] = o[2] = o[3] = 0.0;
                    continue;
                }
                const double* vc = J->grid + c0 * 3;
                double di[3], dj[3];
                /* derivative along i (columns) */
                size_t cl = c0 - 1, cr = c0 + 1, cu = c0 - GW, cd = c0 + GW;
                for (int c = 0; c < 3; ++c) {
                    if (J->gvalid[cl] && J->gvalid[cr])
                        di[c] = (J->grid[cr * 3 + c] - J->grid[cl * 3 + c]) * 0.5;
                    else if (J->gvalid[cr])
                        di[c] = J->grid[cr * 3 + c] - vc[c];
                    else if (J->gvalid[cl])
                        di[c] = vc[c] - J->grid[cl * 3 + c];
                    else
                        di[c] = 0.0;
                    if (J->gvalid[cu] && J->gvalid[cd])
                        dj[c] = (J->grid[cd * 3 + c] - J->grid[cu * 3 + c]) * 0.5;
                    else if (J->gvalid[cd])
                        dj[c] = J->grid[cd * 3 + c] - vc[c];
                    else if (J->gvalid[cu])
                        dj[c] = vc[c] - J->grid[cu * 3 + c];
                    else
                        dj[c] = 0.0;
                }
                double fw = 0.0;
                for (int c = 0; c < 3; ++c) {
                    double f = fabs(di[c]) + fabs(dj[c]);
                    if (f > fw) fw = f;
                }
                if (fw > 0.0) {
                    o[0] = vc[0];
                    o[1] = vc[1];
                    o[2] = vc[2];
                    o[3] = 1.0 / fw;
                } else {
                    o[0] = o[1] = o[2] = o[3] = 0.0;
                }
            }
        }
    }
    return NULL;
}

static int ncores(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

static void run_threads(int n, void* (*fn)(void*), void* arg)
{
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n);
    for (int t = 0; t < n; ++t) pthread_create(&th[t], NULL, fn, arg);
    for (int t = 0; t < n; ++t) pthread_join(th[t], NULL);
    free(th);
}

int orc_map(int W, int H, const double* p, int aov, double* out, int nthreads)
{
    if (W <= 0 || H <= 0) return -1;
    size_t gn = (size_t)(W + 2) * (size_t)(H + 2);
    map_job J;
    J.W = W;
    J.H = H;
    J.aov = aov;
    J.p = p;
    J.grid = (double*)malloc(gn * 3 * sizeof(double));
    J.gvalid = (int*)malloc(gn * sizeof(int));
    J.out = out;
    if (!J.grid || !J.gvalid) {
        free(J.grid);
        free(J.gvalid);
        return -2;
    }
    int n = ncores(nthreads);
    J.phase = 0;
    J.next_row = 0;
    run_threads(n, map_worker, &J);
    J.phase = 1;
    J.next_row = 0;
    run_threads(n, map_worker, &J);
    free(J.grid);
    free(J.gvalid);
    return 0;
}

/* ------------------------------------------------------------------------
 * Triangle setup.
 *
 * Camera: cam = {O_x, O_y, O_z, M (3x3 row-major)}; camera-space vertex
 * X' = M (X - O).
 *
 * Edge normals (Sec. 1.1): n_AB = sigma ||A' x B'||, n_BC, n_CA with
 * sigma = sign(A'.(B' x C')) (reading R10).  The cross product of each edge
 * is formed with the edge's vertices in canonical order and negated when the
 * triangle lists them the other way (reading R11).
 *
 * Miter (Sec. 1.1.2): with A-hat, B-hat, C-hat the normalised vertices,
 *   a^2 = |B-C|^2, b^2 = |C-A|^2, c^2 = |A-B|^2,
 *   O_s = a^2(b^2+c^2-a^2), O_t = b^2(c^2+a^2-b^2), O_p = c^2(a^2+b^2-c^2),
 *   S = (B+C)/2 if O_s <= 0, else (C+A)/2 if O_t <= 0, else (A+B)/2 if
 *   O_p <= 0, else (O_s A + O_t B + O_p C)/(O_s+O_t+O_p);
 *   stored as S-hat, |S| = cos(rho) and sin(rho) = sqrt(1 - |S|^2).
 *
 * Plane (Sec. 1.1.4): N = (A'-B') x (C'-B'), d = A'.N.
 *
 * Culled (valid = 0): a vertex at the eye, A'.(B' x C') == 0, or a cap whose
 * sin(rho) rounds to zero (a triangle far below a pixel).
 */
/* Canonical vertex order: lexicographic order of the bit patterns of the
 * world coordinates (FP32 patterns for FP32 input; the FP64 patterns of
 * FP32 values promoted to double order the same way). */
static int vertex_less_f(const float* P, const float* Q)
{
    for (int c = 0; c < 3; ++c) {
        uint32_t a, b;
        memcpy(&a, &P[c], 4);
        memcpy(&b, &Q[c], 4);
        if (a != b) return a < b;
    }
    return 0;
}

static int vertex_less_d(const double* P, const double* Q)
{
    for (int c = 0; c < 3; ++c) {
        uint64_t a, b;
        memcpy(&a, &P[c], 8);
        memcpy(&b, &Q[c], 8);
        if (a != b) return a < b;
    }
    return 0;
}

static void edge_normal(int swap, const double* Pc, const double* Qc, double sigma, double* n)
{
    double x[3];
    if (swap) {
        /* canonical order is (Q, P): n = -(Q' x P') */
        cross3(Qc, Pc, x);
        x[0] = -x[0];
        x[1] = -x[1];
        x[2] = -x[2];
    } else {
        cross3(Pc, Qc, x);
    }
    double len = sqrt(dot3(x, x));
    for (int c = 0; c < 3; ++c) n[c] = sigma * x[c] / len;
}

/* One triangle: w = world vertices A, B, C (double); swap[e] = 1 when edge
 * e = AB, BC, CA lists its vertices against the canonical order. */
static void setup_one(const double* w, const int* swap, const double* O, const double* M, double* r)
{
    memset(r, 0, sizeof(double) * ORC_REC);
    double V[3][3];
    int at_eye = 0;
    for (int q = 0; q < 3; ++q) {
        double d[3] = {w[3 * q] - O[0], w[3 * q + 1] - O[1], w[3 * q + 2] - O[2]};
        for (int c = 0; c < 3; ++c) V[q][c] = M[3 * c] * d[0] + M[3 * c + 1] * d[1] + M[3 * c + 2] * d[2];
        if (V[q][0] == 0.0 && V[q][1] == 0.0 && V[q][2] == 0.0) at_eye = 1;
    }
    double bxc[3];
    cross3(V[1], V[2], bxc);
    double det = dot3(V[0], bxc);
    if (at_eye || det == 0.0 || !isfinite(det)) return; /* culled */
    double sigma = det > 0.0 ? 1.0 : -1.0;
    edge_normal(swap[0], V[0], V[1], sigma, r + REC_N1);
    edge_normal(swap[1], V[1], V[2], sigma, r + REC_N2);
    edge_normal(swap[2], V[2], V[0], sigma, r + REC_N3);

    /* miter: smallest circle over the projected vertices */
    double U[3][3];
    for (int q = 0; q < 3; ++q) {
        double len = sqrt(dot3(V[q], V[q]));
        for (int c = 0; c < 3; ++c) U[q][c] = V[q][c] / len;
    }
    double e_a[3], e_b[3], e_c[3];
    for (int c = 0; c < 3; ++c) {
        e_a[c] = U[1][c] - U[2][c];
        e_b[c] = U[2][c] - U[0][c];
        e_c[c] = U[0][c] - U[1][c];
    }
    double a2 = dot3(e_a, e_a), b2 = dot3(e_b, e_b), c2 = dot3(e_c, e_c);
    double Os = a2 * (b2 + c2 - a2), Ot = b2 * (c2 + a2 - b2), Op = c2 * (a2 + b2 - c2);
    double S[3];
    for (int c = 0; c < 3; ++c) {
        if (Os <= 0.0)
            S[c] = 0.5 * (U[1][c] + U[2][c]);
        else if (Ot <= 0.0)
            S[c] = 0.5 * (U[2][c] + U[0][c]);
        else if (Op <= 0.0)
            S[c] = 0.5 * (U[0][c] + U[1][c]);
        else
            S[c] = (Os * U[0][c] + Ot * U[1][c] + Op * U[2][c]) / (Os + Ot + Op);
    }
    double slen = sqrt(dot3(S, S));
    double sr = sqrt((1.0 - slen) * (1.0 + slen)); /* sin(rho), reading R17 */
    if (!(slen > 0.0) || !(sr > 0.0)) return; /* degenerate: det == 0, or a point-sized cap */
    for (int c = 0; c < 3; ++c) r[REC_S + c] = S[c] / slen;
    r[REC_C] = slen;
    r[REC_SR] = sr;

    /* plane for depth */
    double ab[3], cb[3];
    for (int c = 0; c < 3; ++c) {
        ab[c] = V[0][c] - V[1][c];
        cb[c] = V[2][c] - V[1][c];
    }
    cross3(ab, cb, r + REC_N);
    r[REC_D] = dot3(V[0], r + REC_N);
    r[REC_VALID] = 1.0;
    r[REC_SIGMA] = sigma;
}

void orc_setup(int64_t T, const float* tris, const float* cam, double* rec)
{
    const double O[3] = {cam[0], cam[1], cam[2]};
    double M[9];
    for (int q = 0; q < 9; ++q) M[q] = cam[3 + q];
    for (int64_t t = 0; t < T; ++t) {
        const float* w = tris + 9 * t;
        double wd[9];
        for (int q = 0; q < 9; ++q) wd[q] = w[q];
        int swap[3] = {vertex_less_f(w + 3, w + 0), vertex_less_f(w + 6, w + 3), vertex_less_f(w + 0, w + 6)};
        setup_one(wd, swap, O, M, rec + ORC_REC * t);
    }
}

/* The same set-up from double-precision world vertices and camera (used to
 * differentiate by central differences with steps far below an FP32 ulp). */
void orc_setup64(int64_t T, const double* tris, const double* cam, double* rec)
{
    const double O[3] = {cam[0], cam[1], cam[2]};
    double M[9];
    for (int q = 0; q < 9; ++q) M[q] = cam[3 + q];
    for (int64_t t = 0; t < T; ++t) {
        const double* w = tris + 9 * t;
        int swap[3] = {vertex_less_d(w + 3, w + 0), vertex_less_d(w + 6, w + 3), vertex_less_d(w + 0, w + 6)};
        setup_one(w, swap, O, M, rec + ORC_REC * t);
    }
}

/* ------------------------------------------------------------------------
 * Rasterization of one pixel against every triangle.
 *
 * For pixel direction G and global delta delta:
 *   g_1..3 = G . n_i, g_4 = (G . S-hat - |S|) / sin(rho)
 *                                   (eq. "rasterization"; reading R17)
 *   fragment  iff  g_i > -1/(2 delta) for all four (gbpxstep) and r > 0
 *   m^f       = min_i clamp(delta g_i + 1/2, 0, 1)        (gpstep, min)
 *   r         = d / (G . N)                               (depth)
 *   centre-inside iff bstep on g_1..3 with the tie rule R11
 * Fragments are merged front to back in ascending (r, t)  (reading R15):
 *   m^fc = min(m^f, 1 - m^b);  m^b = m^b + m^fc          (Sec. 1.4)
 * cov = final m^b; id, depth = the first centre-inside fragment.
 */
typedef struct {
    double r, m;
    uint32_t t;
    int inside;
} frag;

static int frag_cmp(const void* a, const void* b)
{
    const frag* x = (const frag*)a;
    const frag* y = (const frag*)b;
    if (x->r < y->r) return -1;
    if (x->r > y->r) return 1;
    return x->t < y->t ? -1 : (x->t > y->t ? 1 : 0);
}

static int tie_inside(double g, const double* n)
{
    if (g > 0.0) return 1;
    if (g < 0.0) return 0;
    /* g == 0: perturbed sample (eps, eps^2, eps^3) */
    for (int c = 0; c < 3; ++c) {
        if (n[c] > 0.0) return 1;
        if (n[c] < 0.0) return 0;
    }
    return 0;
}

typedef struct {
    int W, H;
    const double* map;
    const double* dmap; /* per-pixel (d_i G, d_j G) for pstep, NULL for gpstep */
    int64_t T;
    const double* rec;
    int64_t npix;
    const int64_t* pix;
    uint32_t* id;
    double* depth;
    double* cov;
    double* sum_mf;
    int32_t* n_inside;
    int32_t* n_frag;
    int64_t next;
    int64_t n_alg;
} raster_job;

static void* raster_worker(void* arg)
{
    raster_job* J = (raster_job*)arg;
    size_t cap = 64;
    frag* F = (frag*)malloc(cap * sizeof(frag));
    int64_t n_alg = 0;
    const int64_t chunk = 64;
    for (;;) {
        int64_t q0 = __atomic_fetch_add(&J->next, chunk, __ATOMIC_RELAXED);
        if (q0 >= J->npix) break;
        int64_t q1 = q0 + chunk < J->npix ? q0 + chunk : J->npix;
        for (int64_t q = q0; q < q1; ++q) {
            int64_t p = J->pix ? J->pix[q] : q;
            const double* G = J->map + 4 * p;
            double delta = G[3];
            size_t nf = 0;
            if (delta > 0.0) {
                double lim = -0.5 / delta;
                const double* dI = J->dmap ? J->dmap + 6 * p : NULL;
                const double* dJ = J->dmap ? J->dmap + 6 * p + 3 : NULL;
                for (int64_t t = 0; t < J->T; ++t) {
                    const double* r = J->rec + ORC_REC * t;
                    if (r[REC_VALID] == 0.0) continue;
                    double g4 = (dot3(G, r + REC_S) - r[REC_C]) / r[REC_SR];
                    /* pstep (Sec. 1.1.1): the ramp of each distance is its own
                     * fwidth, |d_i g| + |d_j g| with d g = n . d G (reading R29) */
                    double w4 = 0.0, w[3] = {0.0, 0.0, 0.0};
                    if (dI) {
                        w4 = (fabs(dot3(r + REC_S, dI)) + fabs(dot3(r + REC_S, dJ))) / r[REC_SR];
                        for (int e = 0; e < 3; ++e)
                            w[e] = fabs(dot3(r + REC_N1 + 3 * e, dI)) + fabs(dot3(r + REC_N1 + 3 * e, dJ));
                        if (!(g4 > -0.5 * w4)) continue;
                    } else if (!(g4 > lim)) {
                        continue;
                    }
                    ++n_alg; /* G inside the enlarged cap: one algorithmic test */
                    double g1 = dot3(G, r + REC_N1), g2 = dot3(G, r + REC_N2), g3 = dot3(G, r + REC_N3);
                    if (dI) {
                        if (!(g1 > -0.5 * w[0] && g2 > -0.5 * w[1] && g3 > -0.5 * w[2])) continue;
                    } else if (!(g1 > lim && g2 > lim && g3 > lim)) {
                        continue;
                    }
                    double rr = r[REC_D] / dot3(G, r + REC_N);
                    if (!(rr > 0.0) || !isfinite(rr)) continue;
                    double m = 1.0;
                    double gs[4] = {g1, g2, g3, g4};
                    double ws[4] = {w[0], w[1], w[2], w4};
                    for (int i = 0; i < 4; ++i) {
                        double st = dI ? clampd(gs[i] / fmax(ws[i], 1e-300) + 0.5, 0.0, 1.0)
                                       : clampd(delta * gs[i] + 0.5, 0.0, 1.0);
                        if (st < m) m = st;
                    }
                    if (nf == cap) {
                        cap *= 2;
                        F = (frag*)realloc(F, cap * sizeof(frag));
                    }
                    F[nf].r = rr;
                    F[nf].m = m;
                    F[nf].t = (uint32_t)t;
                    F[nf].inside = tie_inside(g1, r + REC_N1) && tie_inside(g2, r + REC_N2) &&
                                   tie_inside(g3, r + REC_N3);
                    ++nf;
                }
            }
            qsort(F, nf, sizeof(frag), frag_cmp);
            double mb = 0.0, sum = 0.0;
            uint32_t best = 0xFFFFFFFFu;
            double bdepth = INFINITY;
            int32_t ninside = 0;
            for (size_t f = 0; f < nf; ++f) {
                double mfc = F[f].m < 1.0 - mb ? F[f].m : 1.0 - mb;
                mb = mb + mfc;
                sum += F[f].m;
                if (F[f].inside) {
                    if (ninside == 0) {
                        best = F[f].t;
                        bdepth = F[f].r;
                    }
                    ++ninside;
                }
            }
            J->id[q] = best;
            J->depth[q] = bdepth;
            J->cov[q] = mb;
            if (J->sum_mf) J->sum_mf[q] = sum;
            if (J->n_inside) J->n_inside[q] = ninside;
            if (J->n_frag) J->n_frag[q] = (int32_t)nf;
        }
    }
    free(F);
    __atomic_fetch_add(&J->n_alg, n_alg, __ATOMIC_RELAXED);
    return NULL;
}

/* map: H*W*4 doubles; rec: T*ORC_REC; pix: npix pixel indices (j*W+i) or
 * NULL for all pixels in order (then npix must be W*H).  Outputs have npix
 * entries; sum_mf, n_inside, n_frag may be NULL.  Returns the number of
 * algorithmic tests (pairs inside the enlarged cap), or -1 on bad sizes. */
int64_t orc_raster(int W, int H, const double* map, int64_t T, const double* rec, int64_t npix,
                   const int64_t* pix, uint32_t* id, double* depth, double* cov, double* sum_mf,
                   int32_t* n_inside, int32_t* n_frag, int nthreads)
{
    if (W <= 0 || H <= 0 || T < 0 || npix < 0) return -1;
    if (!pix && npix != (int64_t)W * H) return -1;
    raster_job J;
    J.W = W;
    J.H = H;
    J.map = map;
    J.dmap = NULL;
    J.T = T;
    J.rec = rec;
    J.npix = npix;
    J.pix = pix;
    J.id = id;
    J.depth = depth;
    J.cov = cov;
    J.sum_mf = sum_mf;
    J.n_inside = n_inside;
    J.n_frag = n_frag;
    J.next = 0;
    J.n_alg = 0;
    run_threads(ncores(nthreads), raster_worker, &J);
    return J.n_alg;
}

/* The same rasterization with the per-fragment pixel step (pstep, Sec.
 * 1.1.1) instead of the global delta: m^f = min_i clamp(g_i / w_i + 1/2,
 * 0, 1), fragment iff every g_i > -w_i / 2, with w_i = |d_i g_i| + |d_j g_i|
 * the fwidth of each distance, d g = n . d G for the edge planes and
 * (S-hat . d G) / sin(rho) for the miter (reading R29).  dmap: H*W*6
 * doubles, (d_i G, d_j G) per pixel (orc_map_derivs).  map's 4th channel
 * only marks valid pixels (delta > 0). */
int64_t orc_raster_pstep(int W, int H, const double* map, const double* dmap, int64_t T, const double* rec,
                         int64_t npix, const int64_t* pix, uint32_t* id, double* depth, double* cov, double* sum_mf,
                         int32_t* n_inside, int32_t* n_frag, int nthreads)
{
    if (W <= 0 || H <= 0 || T < 0 || npix < 0 || !dmap) return -1;
    if (!pix && npix != (int64_t)W * H) return -1;
    raster_job J;
    J.W = W;
    J.H = H;
    J.map = map;
    J.dmap = dmap;
    J.T = T;
    J.rec = rec;
    J.npix = npix;
    J.pix = pix;
    J.id = id;
    J.depth = depth;
    J.cov = cov;
    J.sum_mf = sum_mf;
    J.n_inside = n_inside;
    J.n_frag = n_frag;
    J.next = 0;
    J.n_alg = 0;
    run_threads(ncores(nthreads), raster_worker, &J);
    return J.n_alg;
}

/* ------------------------------------------------------------------------
 * Shaded image (the differentiable workload): per pixel the front-to-back
 * merge of Sec. 1.4 applied to a shade pass, as the paper applies it to its
 * depth, UV and normal passes:
 *   m^fc = min(m^f, 1 - m^b);  I = I + m^fc * shade_f;  m^b = m^b + m^fc
 * over the fragments in ascending (r, t), with shade_f = c_t |N-hat_t . G|
 * (a Lambert-like term of the triangle's unit plane normal).  Fragments and
 * m^f as in orc_raster.  image: npix values.
 */
typedef struct {
    double r, m, shade;
    uint32_t t;
} sfrag;

static int sfrag_cmp(const void* a, const void* b)
{
    const sfrag* x = (const sfrag*)a;
    const sfrag* y = (const sfrag*)b;
    if (x->r < y->r) return -1;
    if (x->r > y->r) return 1;
    return x->t < y->t ? -1 : (x->t > y->t ? 1 : 0);
}

typedef struct {
    int W, H;
    const double* map;
    int64_t T;
    const double* rec;
    const double* colors;
    int64_t npix;
    const int64_t* pix;
    double* image;
    int64_t next;
} shade_job;

static void* shade_worker(void* arg)
{
    shade_job* J = (shade_job*)arg;
    size_t cap = 64;
    sfrag* F = (sfrag*)malloc(cap * sizeof(sfrag));
    for (;;) {
        int64_t q0 = __atomic_fetch_add(&J->next, 64, __ATOMIC_RELAXED);
        if (q0 >= J->npix) break;
        int64_t q1 = q0 + 64 < J->npix ? q0 + 64 : J->npix;
        for (int64_t q = q0; q < q1; ++q) {
            int64_t p = J->pix ? J->pix[q] : q;
            const double* G = J->map + 4 * p;
            double delta = G[3];
            size_t nf = 0;
            if (delta > 0.0) {
                double lim = -0.5 / delta;
                for (int64_t t = 0; t < J->T; ++t) {
                    const double* r = J->rec + ORC_REC * t;
                    if (r[REC_VALID] == 0.0) continue;
                    double g4 = (dot3(G, r + REC_S) - r[REC_C]) / r[REC_SR];
                    if (!(g4 > lim)) continue;
                    double g1 = dot3(G, r + REC_N1), g2 = dot3(G, r + REC_N2), g3 = dot3(G, r + REC_N3);
                    if (!(g1 > lim && g2 > lim && g3 > lim)) continue;
                    double GN = dot3(G, r + REC_N);
                    double rr = r[REC_D] / GN;
                    if (!(rr > 0.0) || !isfinite(rr)) continue;
                    double m = 1.0;
                    double gs[4] = {g1, g2, g3, g4};
                    for (int i = 0; i < 4; ++i) {
                        double st = clampd(delta * gs[i] + 0.5, 0.0, 1.0);
                        if (st < m) m = st;
                    }
                    if (nf == cap) {
                        cap *= 2;
                        F = (sfrag*)realloc(F, cap * sizeof(sfrag));
                    }
                    double nlen = sqrt(dot3(r + REC_N, r + REC_N));
                    F[nf].r = rr;
                    F[nf].m = m;
                    F[nf].shade = J->colors[t] * fabs(GN / nlen);
                    F[nf].t = (uint32_t)t;
                    ++nf;
                }
            }
            qsort(F, nf, sizeof(sfrag), sfrag_cmp);
            double mb = 0.0, img = 0.0;
            for (size_t f = 0; f < nf; ++f) {
                double mfc = F[f].m < 1.0 - mb ? F[f].m : 1.0 - mb;
                img += mfc * F[f].shade;
                mb += mfc;
            }
            J->image[q] = img;
        }
    }
    free(F);
    return NULL;
}

int orc_shade(int W, int H, const double* map, int64_t T, const double* rec, const double* colors, int64_t npix,
              const int64_t* pix, double* image, int nthreads)
{
    if (W <= 0 || H <= 0 || T < 0 || npix < 0) return -1;
    if (!pix && npix != (int64_t)W * H) return -1;
    shade_job J = {W, H, map, T, rec, colors, npix, pix, image, 0};
    run_threads(ncores(nthreads), shade_worker, &J);
    return 0;
}

/* ------------------------------------------------------------------------
 * Derivatives of the map with respect to the lens parameters
 * (k, l, s, Omega in degrees), by the complex-step method (Squire and
 * Trapp 1998): the map function is analytic in each parameter, so with the
 * parameter p_j + i h, h = 1e-30, Im v / h is dv/dp_j to the last bit, with
 * no subtractive cancellation.  delta = 1/fw with fw = max_c (|d_i v_c| +
 * |d_j v_c|) (reading R8) is differentiated by the chain rule at the
 * maximising component (the first one, as in orc_map) and the signs of its
 * differences.  out[(j*W + i)*4 + 0..3] = (dv_x, dv_y, dv_z, d delta)/dp_j;
 * zero on invalid pixels.  which: 0 k, 1 l, 2 s, 3 Omega.
 */
#include <complex.h>

static int map_dir_cs(double x, double y, const double* p, int which, double* v, double* dv)
{
    const double h = 1e-30;
    double complex k = p[0], l = p[1], s = p[2], om = p[3];
    if (which == 0) k += I * h;
    if (which == 1) l += I * h;
    if (which == 2) s += I * h;
    if (which == 3) om += I * h;
    double complex half = om * ORC_PI / 360.0;
    double complex R = csqrt(x * x + l * y * y);
    double complex theta, sor;
    int Rzero = x == 0.0 && y == 0.0;
    if (p[0] > 0.0) {
        double complex tk = ctan(k * half);
        theta = catan(tk * R) / k;
        sor = Rzero ? tk / k : csin(theta) / R;
    } else if (p[0] == 0.0) {
        theta = half * R;
        sor = Rzero ? half : csin(theta) / R;
    } else {
        double complex sk = csin(k * half);
        double complex arg = sk * R;
        if (creal(arg) > 1.0 || creal(arg) < -1.0) {
            v[0] = v[1] = v[2] = dv[0] = dv[1] = dv[2] = 0.0;
            return 0;
        }
        theta = casin(arg) / k;
        sor = Rzero ? sk / k : csin(theta) / R;
    }
    double complex w[3] = {x * sor, y * sor / (l * (1.0 - s) + s), ccos(theta)};
    double complex n = csqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int c = 0; c < 3; ++c) {
        double complex q = w[c] / n;
        v[c] = creal(q);
        dv[c] = cimag(q) / h;
    }
    return 1;
}

int orc_map_tangent(int W, int H, const double* p, int aov, int which, double* out)
{
    if (W <= 0 || H <= 0 || which < 0 || which > 3) return -1;
    const int GW = W + 2;
    const size_t gn = (size_t)GW * (size_t)(H + 2);
    double* g = (double*)malloc(gn * 6 * sizeof(double));
    int* ok = (int*)malloc(gn * sizeof(int));
    if (!g || !ok) {
        free(g);
        free(ok);
        return -2;
    }
    const double aspect = (double)W / (double)H;
    for (int gj = 0; gj < H + 2; ++gj)
        for (int gi = 0; gi < GW; ++gi) {
            size_t q = (size_t)gj * GW + gi;
            double xy[2];
            orc_view_coord((gi - 0.5) / W, (gj - 0.5) / H, aspect, aov, xy);
            ok[q] = map_dir_cs(xy[0], xy[1], p, which, g + 6 * q, g + 6 * q + 3);
        }
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double* o = out + ((size_t)j * W + i) * 4;
            size_t c0 = (size_t)(j + 1) * GW + (i + 1);
            o[0] = o[1] = o[2] = o[3] = 0.0;
            if (!ok[c0]) continue;
            size_t cl = c0 - 1, cr = c0 + 1, cu = c0 - GW, cd = c0 + GW;
            double fw = 0.0, dfw = 0.0;
            for (int c = 0; c < 3; ++c) {
                /* value (0) and tangent (3) of the two differences */
                double di[2], dj[2];
                for (int part = 0; part < 2; ++part) {
                    int off = part ? 3 : 0;
                    double vc = g[6 * c0 + off + c];
                    if (ok[cl] && ok[cr])
                        di[part] = (g[6 * cr + off + c] - g[6 * cl + off + c]) * 0.5;
                    else if (ok[cr])
                        di[part] = g[6 * cr + off + c] - vc;
                    else if (ok[cl])
                        di[part] = vc - g[6 * cl + off + c];
                    else
                        di[part] = 0.0;
                    if (ok[cu] && ok[cd])
                        dj[part] = (g[6 * cd + off + c] - g[6 * cu + off + c]) * 0.5;
                    else if (ok[cd])
                        dj[part] = g[6 * cd + off + c] - vc;
                    else if (ok[cu])
                        dj[part] = vc - g[6 * cu + off + c];
                    else
                        dj[part] = 0.0;
                }
                double f = fabs(di[0]) + fabs(dj[0]);
                if (f > fw) {
                    fw = f;
                    double si = di[0] > 0.0 ? 1.0 : (di[0] < 0.0 ? -1.0 : 0.0);
                    double sj = dj[0] > 0.0 ? 1.0 : (dj[0] < 0.0 ? -1.0 : 0.0);
                    dfw = si * di[1] + sj * dj[1];
                }
            }
            if (!(fw > 0.0)) continue;
            for (int c = 0; c < 3; ++c) o[c] = g[6 * c0 + 3 + c];
            o[3] = -dfw / (fw * fw);
        }
    free(g);
    free(ok);
    return 0;
}

/* ------------------------------------------------------------------------
 * Adjoint of the shaded image (and of the coverage and depth outputs) with
 * respect to the set-up records, the colours and the map, per pixel in the
 * merge order of orc_shade.  With upstream gradients dI, dcov, ddepth of a
 * pixel and its fragments f = 0, 1, ... in ascending (r, t):
 *
 *   the merge m^fc = min(m^f, 1 - m^b), m^b += m^fc takes m^fc = m^f until
 *   the first fragment f* with m^f > 1 - m^b, which takes 1 - m^b and
 *   leaves m^b = 1 (every later fragment then adds nothing).  Hence
 *     dI/d shade_f = m^fc_f,
 *     dI/d m^f_f   = shade_f - shade_f*  for f < f* (shade_f alone when no
 *                    fragment saturates the pixel), 0 from f* on,
 *     dcov/d m^f_f = 1 for every f when no fragment saturates, else 0;
 *   m^f = min_i clamp(delta g_i + 1/2, 0, 1) passes its gradient to the
 *   first minimising distance i* when its clamp is not saturated:
 *     d g_i* = delta dm, d delta = g_i* dm;
 *   g_1..3 = G.n_i, g_4 = (G.S-hat - c)/sin(rho), sin(rho) = sqrt(1 - c^2);
 *   shade = col |G.N|/|N|;  depth r = d/(G.N) of the nearest centre-inside
 *   fragment.
 *
 * drec[t*ORC_REC + ...] receives d/d(n_1, n_2, n_3, S-hat, c, N, d) at the
 * record offsets (REC_N1 .. REC_D); dcolors[t]; dmap[q*4 + 0..3] =
 * d/d(G, delta) of listed pixel q.  Single-threaded over pixels (the
 * accumulation into drec is then in a fixed order).
 */
int orc_shade_grad(int W, int H, const double* map, int64_t T, const double* rec, const double* colors,
                   int64_t npix, const int64_t* pix, const double* dimage, const double* dcov, const double* ddepth,
                   double* drec, double* dcolors, double* dmap)
{
    if (W <= 0 || H <= 0 || T < 0 || npix < 0) return -1;
    if (!pix && npix != (int64_t)W * H) return -1;
    memset(drec, 0, sizeof(double) * ORC_REC * (size_t)T);
    memset(dcolors, 0, sizeof(double) * (size_t)T);
    size_t cap = 64;
    sfrag* F = (sfrag*)malloc(cap * sizeof(sfrag));
    for (int64_t q = 0; q < npix; ++q) {
        int64_t p = pix ? pix[q] : q;
        const double* G = map + 4 * p;
        const double delta = G[3];
        double* dG = dmap + 4 * q;
        dG[0] = dG[1] = dG[2] = dG[3] = 0.0;
        if (!(delta > 0.0)) continue;
        const double lim = -0.5 / delta;
        size_t nf = 0;
        for (int64_t t = 0; t < T; ++t) {
            const double* r = rec + ORC_REC * t;
            if (r[REC_VALID] == 0.0) continue;
            double g4 = (dot3(G, r + REC_S) - r[REC_C]) / r[REC_SR];
            if (!(g4 > lim)) continue;
            double g1 = dot3(G, r + REC_N1), g2 = dot3(G, r + REC_N2), g3 = dot3(G, r + REC_N3);
            if (!(g1 > lim && g2 > lim && g3 > lim)) continue;
            double GN = dot3(G, r + REC_N);
            double rr = r[REC_D] / GN;
            if (!(rr > 0.0) || !isfinite(rr)) continue;
            double m = 1.0;
            double gs[4] = {g1, g2, g3, g4};
            for (int i = 0; i < 4; ++i) {
                double st = clampd(delta * gs[i] + 0.5, 0.0, 1.0);
                if (st < m) m = st;
            }
            if (nf == cap) {
                cap *= 2;
                F = (sfrag*)realloc(F, cap * sizeof(sfrag));
            }
            double nlen = sqrt(dot3(r + REC_N, r + REC_N));
            F[nf].r = rr;
            F[nf].m = m;
            F[nf].shade = colors[t] * fabs(GN / nlen);
            F[nf].t = (uint32_t)t;
            ++nf;
        }
        qsort(F, nf, sizeof(sfrag), sfrag_cmp);
        const double dI = dimage ? dimage[q] : 0.0;
        const double dC = dcov ? dcov[q] : 0.0;
        const double dD = ddepth ? ddepth[q] : 0.0;
        /* the saturating fragment f*, if any */
        size_t fstar = nf;
        double mb = 0.0;
        for (size_t f = 0; f < nf; ++f) {
            if (F[f].m > 1.0 - mb) {
                fstar = f;
                break;
            }
            mb += F[f].m;
        }
        const double beta = fstar < nf ? -dI * F[fstar].shade : dC;
        mb = 0.0;
        const size_t last = fstar < nf ? fstar + 1 : nf;
        for (size_t f = 0; f < last; ++f) {
            const int64_t t = F[f].t;
            const double* r = rec + ORC_REC * t;
            double* dr = drec + ORC_REC * t;
            double dm, dshade;
            if (f == fstar) {
                dm = 0.0;
                dshade = dI * (1.0 - mb);
            } else {
                dm = dI * F[f].shade + beta;
                dshade = dI * F[f].m;
                mb += F[f].m;
            }
            /* m^f: the first minimising distance, if its clamp is open */
            if (dm != 0.0) {
                double gs[4] = {dot3(G, r + REC_N1), dot3(G, r + REC_N2), dot3(G, r + REC_N3),
                                (dot3(G, r + REC_S) - r[REC_C]) / r[REC_SR]};
                double m = 1.0;
                int istar = -1;
                for (int i = 0; i < 4; ++i) {
                    double st = clampd(delta * gs[i] + 0.5, 0.0, 1.0);
                    if (st < m) {
                        m = st;
                        istar = i;
                    }
                }
                double arg = istar >= 0 ? delta * gs[istar] + 0.5 : 1.0;
                if (istar >= 0 && arg > 0.0 && arg < 1.0) {
                    const double dg = dm * delta;
                    dG[3] += dm * gs[istar];
                    if (istar < 3) {
                        const int off = REC_N1 + 3 * istar;
                        for (int c = 0; c < 3; ++c) {
                            dr[off + c] += dg * G[c];
                            dG[c] += dg * r[off + c];
                        }
                    } else {
                        const double sr = r[REC_SR], cc = r[REC_C];
                        for (int c = 0; c < 3; ++c) {
                            dr[REC_S + c] += dg * G[c] / sr;
                            dG[c] += dg * r[REC_S + c] / sr;
                        }
                        dr[REC_C] += dg * (-1.0 / sr + gs[3] * cc / (sr * sr));
                    }
                }
            }
            /* shade = col |G.N| / |N| */
            if (dshade != 0.0) {
                const double nlen = sqrt(dot3(r + REC_N, r + REC_N));
                const double u = dot3(G, r + REC_N) / nlen;
                dcolors[t] += dshade * fabs(u);
                const double du = dshade * colors[t] * (u > 0.0 ? 1.0 : (u < 0.0 ? -1.0 : 0.0));
                for (int c = 0; c < 3; ++c) {
                    dG[c] += du * r[REC_N + c] / nlen;
                    dr[REC_N + c] += du * (G[c] - u * r[REC_N + c] / nlen) / nlen;
                }
            }
        }
        /* depth of the nearest centre-inside fragment */
        if (dD != 0.0) {
            for (size_t f = 0; f < nf; ++f) {
                const double* r = rec + ORC_REC * F[f].t;
                if (!(tie_inside(dot3(G, r + REC_N1), r + REC_N1) && tie_inside(dot3(G, r + REC_N2), r + REC_N2) &&
                      tie_inside(dot3(G, r + REC_N3), r + REC_N3)))
                    continue;
                double* dr = drec + ORC_REC * F[f].t;
                const double GN = dot3(G, r + REC_N);
                dr[REC_D] += dD / GN;
                const double dGN = -dD * F[f].r / GN;
                for (int c = 0; c < 3; ++c) {
                    dG[c] += dGN * r[REC_N + c];
                    dr[REC_N + c] += dGN * G[c];
                }
                break;
            }
        }
    }
    free(F);
    return 0;
}

/* ------------------------------------------------------------------------
 * Adjoint of the set-up (orc_setup64's arithmetic, in reverse): record
 * gradients drec (layout of orc_shade_grad) -> world-vertex gradients
 * dtris[t*9 + 3*v + c].
 *   n_e = sigma x/|x|, x = P' x Q'    =>  dx = sigma (dn - x^ (x^.dn))/|x|,
 *                                          dP' += Q' x dx, dQ' += dx x P'
 *   S-hat = S/|S|, c = |S|             =>  dS = (dS^ - S^ (S^.dS^))/|S| + S^ dc
 *   S = (U_a + U_b)/2 or (Os U0 + Ot U1 + Op U2)/(Os + Ot + Op) with the
 *   squared chords a2, b2, c2 of the unit vertices U = V/|V|
 *   N = (A' - B') x (C' - B'), d = A'.N
 *   X' = M (X - O)                     =>  dX = M^T dX'
 */
void orc_setup_grad(int64_t T, const double* tris, const double* cam, const double* rec, const double* drec,
                    double* dtris)
{
    const double O[3] = {cam[0], cam[1], cam[2]};
    const double* M = cam + 3;
    for (int64_t t = 0; t < T; ++t) {
        const double* w = tris + 9 * t;
        const double* r = rec + ORC_REC * t;
        const double* dr = drec + ORC_REC * t;
        double* dw = dtris + 9 * t;
        for (int q = 0; q < 9; ++q) dw[q] = 0.0;
        if (r[REC_VALID] == 0.0) continue;
        double V[3][3], dV[3][3] = {{0}};
        for (int q = 0; q < 3; ++q) {
            double d[3] = {w[3 * q] - O[0], w[3 * q + 1] - O[1], w[3 * q + 2] - O[2]};
            for (int c = 0; c < 3; ++c) V[q][c] = M[3 * c] * d[0] + M[3 * c + 1] * d[1] + M[3 * c + 2] * d[2];
        }
        const double sigma = r[REC_SIGMA];
        /* edge normals */
        for (int e = 0; e < 3; ++e) {
            const int P = e, Q = (e + 1) % 3;
            double x[3];
            cross3(V[P], V[Q], x);
            const double len = sqrt(dot3(x, x));
            const double* dn = dr + REC_N1 + 3 * e;
            double xh[3] = {x[0] / len, x[1] / len, x[2] / len};
            const double pr = dot3(xh, dn);
            double dx[3], a[3], b[3];
            for (int c = 0; c < 3; ++c) dx[c] = sigma * (dn[c] - xh[c] * pr) / len;
            cross3(V[Q], dx, a);
            cross3(dx, V[P], b);
            for (int c = 0; c < 3; ++c) {
                dV[P][c] += a[c];
                dV[Q][c] += b[c];
            }
        }
        /* miter */
        double U[3][3], Ulen[3];
        for (int q = 0; q < 3; ++q) {
            Ulen[q] = sqrt(dot3(V[q], V[q]));
            for (int c = 0; c < 3; ++c) U[q][c] = V[q][c] / Ulen[q];
        }
        double e_a[3], e_b[3], e_c[3];
        for (int c = 0; c < 3; ++c) {
            e_a[c] = U[1][c] - U[2][c];
            e_b[c] = U[2][c] - U[0][c];
            e_c[c] = U[0][c] - U[1][c];
        }
        const double a2 = dot3(e_a, e_a), b2 = dot3(e_b, e_b), c2 = dot3(e_c, e_c);
        const double Os = a2 * (b2 + c2 - a2), Ot = b2 * (c2 + a2 - b2), Op = c2 * (a2 + b2 - c2);
        const double* Sh = r + REC_S;
        const double slen = r[REC_C];
        double S[3], dS[3], dU[3][3] = {{0}};
        for (int c = 0; c < 3; ++c) S[c] = Sh[c] * slen;
        const double prS = dot3(Sh, dr + REC_S);
        for (int c = 0; c < 3; ++c) dS[c] = (dr[REC_S + c] - Sh[c] * prS) / slen + Sh[c] * dr[REC_C];
        if (Os <= 0.0 || Ot <= 0.0 || Op <= 0.0) {
            const int a = Os <= 0.0 ? 1 : (Ot <= 0.0 ? 2 : 0);
            const int b = Os <= 0.0 ? 2 : (Ot <= 0.0 ? 0 : 1);
            for (int c = 0; c < 3; ++c) {
                dU[a][c] += 0.5 * dS[c];
                dU[b][c] += 0.5 * dS[c];
            }
        } else {
            const double sum = Os + Ot + Op;
            const double Oq[3] = {Os, Ot, Op};
            double dO[3];
            for (int q = 0; q < 3; ++q) {
                double u[3] = {U[q][0] - S[0], U[q][1] - S[1], U[q][2] - S[2]};
                dO[q] = dot3(dS, u) / sum;
                for (int c = 0; c < 3; ++c) dU[q][c] += Oq[q] / sum * dS[c];
            }
            const double da2 = dO[0] * (b2 + c2 - 2.0 * a2) + dO[1] * b2 + dO[2] * c2;
            const double db2 = dO[0] * a2 + dO[1] * (c2 + a2 - 2.0 * b2) + dO[2] * c2;
            const double dc2 = dO[0] * a2 + dO[1] * b2 + dO[2] * (a2 + b2 - 2.0 * c2);
            for (int c = 0; c < 3; ++c) {
                dU[1][c] += 2.0 * da2 * e_a[c];
                dU[2][c] -= 2.0 * da2 * e_a[c];
                dU[2][c] += 2.0 * db2 * e_b[c];
                dU[0][c] -= 2.0 * db2 * e_b[c];
                dU[0][c] += 2.0 * dc2 * e_c[c];
                dU[1][c] -= 2.0 * dc2 * e_c[c];
            }
        }
        for (int q = 0; q < 3; ++q) {
            const double pr = dot3(U[q], dU[q]);
            for (int c = 0; c < 3; ++c) dV[q][c] += (dU[q][c] - U[q][c] * pr) / Ulen[q];
        }
        /* plane and depth offset */
        double ab[3], cb[3], N[3];
        for (int c = 0; c < 3; ++c) {
            ab[c] = V[0][c] - V[1][c];
            cb[c] = V[2][c] - V[1][c];
        }
        cross3(ab, cb, N);
        double dN[3];
        for (int c = 0; c < 3; ++c) {
            dN[c] = dr[REC_N + c] + dr[REC_D] * V[0][c];
            dV[0][c] += dr[REC_D] * N[c];
        }
        double de1[3], de2[3];
        cross3(cb, dN, de1);
        cross3(dN, ab, de2);
        for (int c = 0; c < 3; ++c) {
            dV[0][c] += de1[c];
            dV[2][c] += de2[c];
            dV[1][c] -= de1[c] + de2[c];
        }
        /* world */
        for (int q = 0; q < 3; ++q)
            for (int c = 0; c < 3; ++c)
                dw[3 * q + c] = M[c] * dV[q][0] + M[3 + c] * dV[q][1] + M[6 + c] * dV[q][2];
    }
}

/* ------------------------------------------------------------------------
 * Perspective maps of other projections (Sec. 2.2) and the lens distortion
 * of view coordinates (Sec. 2.3), evaluated like orc_map: the direction of
 * every pixel centre, the global delta from central differences of the map
 * function at the neighbouring centres (reading R8), here restricted to
 * neighbours of the same chart (the cube map's faces), invalid pixels
 * (0,0,0,0).
 *
 * kind 0 Universal (param k, l, s, Omega_deg after limits) with the
 *        Brown-Conrady distortion dist[6] = (k1, k2, p1, p2, q1, q2) of its
 *        view coordinates (x, y) in the map's AOV normalisation:
 *        r2 = x^2 + y^2, (x, y) <- (x, y)(1 + k1 r2 + k2 r2^2)
 *                                 + (x, y)(p1 x + p2 y) + (q1, q2) r2
 * kind 1 rectilinear (param Omega_deg): normalize(x, y, cot(Omega/2)),
 *        the same distortion applies
 * kind 2 curved panorama (param Omega_h_deg, height): with
 *        f' = (Omega_h (f_s - 1/2), height (f_t - 1/2)),
 *        v = normalize(sin f'_x, f'_y, cos f'_x)
 * kind 3 full dome (param compression_deg, tilt_deg, offset):
 *        f' = (2 f_s - 1, 1 - 2 f_t), R = |f'|, theta = R (compression + pi/2),
 *        v = normalize(f'_x sin(theta)/R, cos(theta), f'_y sin(theta)/R + offset)
 *        rotated by the tilt about x; pixels with R > 1 are outside the dome
 * kind 4 equirectangular: f' = pi (2 f_s - 1, f_t),
 *        v = (sin f'_x sin f'_y, -cos f'_y, cos f'_x sin f'_y)
 * kind 5 cube map (W = 6 H): face i = floor(6 f_s), local
 *        u = normalize(fract(6 f_s) - 1/2, f_t - 1/2, 1/2), v = M_i u with
 *        the rows of M_i as printed for faces 0, 1, 2, 4, 5 and M_3 = I
 *        (reading: the printed case list has no face 3; the other five look
 *        along +x, -x, -z, +y, -y, so face 3 is the front face along +z)
 */
static int map_spec_dir(double fs, double ft, int W, int H, int kind, const double* prm, const double* dist,
                        int aov, double* v, int* chart)
{
    *chart = 0;
    const double aspect = (double)W / (double)H;
    if (kind == 0 || kind == 1) {
        double xy[2];
        orc_view_coord(fs, ft, aspect, aov, xy);
        double x = xy[0], y = xy[1];
        const double r2 = x * x + y * y;
        const double rad = 1.0 + dist[0] * r2 + dist[1] * r2 * r2;
        const double pr = dist[2] * x + dist[3] * y;
        const double xd = x * rad + x * pr + dist[4] * r2;
        const double yd = y * rad + y * pr + dist[5] * r2;
        if (kind == 0) return orc_map_dir(xd, yd, prm, v);
        double w[3] = {xd, yd, 1.0 / tan(prm[0] * ORC_PI / 360.0)};
        double n = sqrt(dot3(w, w));
        for (int c = 0; c < 3; ++c) v[c] = w[c] / n;
        return 1;
    }
    if (kind == 2) {
        const double fx = prm[0] * ORC_PI / 180.0 * (fs - 0.5), fy = prm[1] * (ft - 0.5);
        double w[3] = {sin(fx), fy, cos(fx)};
        double n = sqrt(dot3(w, w));
        for (int c = 0; c < 3; ++c) v[c] = w[c] / n;
        return 1;
    }
    if (kind == 3) {
        const double fx = 2.0 * fs - 1.0, fy = 1.0 - 2.0 * ft;
        const double R = sqrt(fx * fx + fy * fy);
        if (R > 1.0) {
            v[0] = v[1] = v[2] = 0.0;
            return 0;
        }
        const double theta = R * (prm[0] * ORC_PI / 180.0 + 0.5 * ORC_PI);
        const double sor = R > 0.0 ? sin(theta) / R : prm[0] * ORC_PI / 180.0 + 0.5 * ORC_PI;
        double w[3] = {fx * sor, cos(theta), fy * sor + prm[2]};
        double n = sqrt(dot3(w, w));
        for (int c = 0; c < 3; ++c) w[c] /= n;
        const double ct = cos(prm[1] * ORC_PI / 180.0), st = sin(prm[1] * ORC_PI / 180.0);
        /* row vector times the tilt matrix [[1,0,0],[0,c,-s],[0,s,c]] */
        v[0] = w[0];
        v[1] = w[1] * ct + w[2] * st;
        v[2] = -w[1] * st + w[2] * ct;
        return 1;
    }
    if (kind == 4) {
        const double fx = ORC_PI * (2.0 * fs - 1.0), fy = ORC_PI * ft;
        v[0] = sin(fx) * sin(fy);
        v[1] = -cos(fy);
        v[2] = cos(fx) * sin(fy);
        return 1;
    }
    /* kind 5: cube */
    const double s6 = 6.0 * fs;
    const int face = (int)floor(s6);
    *chart = face;
    if (face < 0 || face > 5) {  /* beyond the strip (halo pixels): no chart */
        v[0] = v[1] = v[2] = 0.0;
        return 0;
    }
    double u[3] = {s6 - face - 0.5, ft - 0.5, 0.5};
    double n = sqrt(dot3(u, u));
    for (int c = 0; c < 3; ++c) u[c] /= n;
    /* rows of M_i: world = M_i u */
    static const double M[6][9] = {
        {0, 0, 1, -1, 0, 0, 0, -1, 0},   /* [ Z, -X, -Y] */
        {0, 0, -1, 1, 0, 0, 0, -1, 0},   /* [-Z,  X, -Y] */
        {1, 0, 0, 0, -1, 0, 0, 0, -1},   /* [ X, -Y, -Z] */
        {1, 0, 0, 0, 1, 0, 0, 0, 1},     /* [ X,  Y,  Z] (reading) */
        {1, 0, 0, 0, 0, 1, 0, -1, 0},    /* [ X,  Z, -Y] */
        {-1, 0, 0, 0, 0, -1, 0, -1, 0},  /* [-X, -Z, -Y] */
    };
    for (int r = 0; r < 3; ++r) v[r] = M[face][3 * r] * u[0] + M[face][3 * r + 1] * u[1] + M[face][3 * r + 2] * u[2];
    return 1;
}

int orc_map_spec(int W, int H, int kind, const double* prm, const double* dist, int aov, double* out, double* deriv)
{
    if (W <= 0 || H <= 0 || kind < 0 || kind > 5) return -1;
    const int GW = W + 2;
    const size_t gn = (size_t)GW * (size_t)(H + 2);
    double* g = (double*)malloc(gn * 3 * sizeof(double));
    int* ok = (int*)malloc(gn * sizeof(int));
    int* ch = (int*)malloc(gn * sizeof(int));
    if (!g || !ok || !ch) {
        free(g);
        free(ok);
        free(ch);
        return -2;
    }
    for (int gj = 0; gj < H + 2; ++gj)
        for (int gi = 0; gi < GW; ++gi) {
            const size_t q = (size_t)gj * GW + gi;
            ok[q] = map_spec_dir((gi - 0.5) / W, (gj - 0.5) / H, W, H, kind, prm, dist, aov, g + 3 * q, &ch[q]);
        }
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            double* o = out + ((size_t)j * W + i) * 4;
            const size_t c0 = (size_t)(j + 1) * GW + (i + 1);
            o[0] = o[1] = o[2] = o[3] = 0.0;
            if (!ok[c0]) continue;
            /* a neighbour counts only when valid and on the same chart */
            const size_t nb[4] = {c0 - 1, c0 + 1, c0 - GW, c0 + GW};
            int use[4];
            for (int q = 0; q < 4; ++q) use[q] = ok[nb[q]] && ch[nb[q]] == ch[c0];
            double fw = 0.0, dv[6];
            for (int c = 0; c < 3; ++c) {
                const double vc = g[3 * c0 + c];
                double di, dj;
                if (use[0] && use[1])
                    di = (g[3 * nb[1] + c] - g[3 * nb[0] + c]) * 0.5;
                else if (use[1])
                    di = g[3 * nb[1] + c] - vc;
                else if (use[0])
                    di = vc - g[3 * nb[0] + c];
                else
                    di = 0.0;
                if (use[2] && use[3])
                    dj = (g[3 * nb[3] + c] - g[3 * nb[2] + c]) * 0.5;
                else if (use[3])
                    dj = g[3 * nb[3] + c] - vc;
                else if (use[2])
                    dj = vc - g[3 * nb[2] + c];
                else
                    dj = 0.0;
                const double f = fabs(di) + fabs(dj);
                if (f > fw) fw = f;
                dv[c] = di;
                dv[3 + c] = dj;
            }
            if (!(fw > 0.0)) continue;
            for (int c = 0; c < 3; ++c) o[c] = g[3 * c0 + c];
            o[3] = 1.0 / fw;
            if (deriv)
                for (int c = 0; c < 6; ++c) deriv[((size_t)j * W + i) * 6 + c] = dv[c];
        }
    free(g);
    free(ok);
    free(ch);
    return 0;
}

/* The map function of orc_map_spec at arbitrary texture coordinates (for
 * the solid-angle pins).  v: n x 3, valid: n. */
void orc_map_spec_dirs(int64_t n, const double* fs, const double* ft, int W, int H, int kind, const double* prm,
                       const double* dist, int aov, double* v, int32_t* valid)
{
    for (int64_t q = 0; q < n; ++q) {
        int chart;
        valid[q] = map_spec_dir(fs[q], ft[q], W, H, kind, prm, dist, aov, v + 3 * q, &chart);
    }
}
