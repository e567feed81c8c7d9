/*
 * FP64 CPU oracle for multiscale sphere tracing, analytic MLP normals and
 * neural normal mapping (da Silva et al., "Neural Implicit Mapping via
 * Nested Neighborhoods", CVPR 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA library; it reads the same SDFN
 * network files with its own parser.
 *
 * Every routine is a plain, slow restatement of the paper in double
 * precision, one ray or point at a time:
 *   oracle_net_eval        Eq. 2            f(p) = W_n . f_{n-1} o ... o f_0(p) + b_n
 *   oracle_net_grad        Alg. 2 / Eqs. 3-4  three independent forward tangent chains
 *   oracle_trace           Alg. 1           multiscale sphere tracing (with the readings below)
 *   oracle_normal_map      Sec. 5           N(p) = grad f(p) at points of a coarse surface
 *   oracle_first_root      (check only)     dense march + bisection for the first root
 *   oracle_lipschitz       (Sec. 4 step bound) product of per-layer spectral norms
 *   oracle_thresholds_*    Sec. 3.3         Props. 1 and 2 threshold recurrences
 *
 * Readings of points the paper leaves open (each mirrored by the CUDA side
 * from its own code):
 *   - Sine frequencies are folded into the weights at load: layer 0 by omega0,
 *     hidden layers by omega; the linear output layer is unchanged.
 *   - Alg. 1 step: t = f_j(p) - d_j (d_j = delta_j, or 0 on the last level
 *     when final_mode == 0); p += s_j * t * v; the level loop runs while
 *     t > eps and fewer than cap_j steps were taken (the paper fixes the
 *     iteration counts, Sec. 6).  The step is taken before the test, as
 *     written in Alg. 1.
 *   - Rays start at their entry into the box [lo, hi]^3 (or at the origin if
 *     it is inside); a ray that misses the box is a miss with no evaluation.
 *     After every step the point must stay inside the box widened by 1e-3,
 *     otherwise the ray is a miss.
 *   - Hit iff the last level's loop ended with t <= eps (it converged) and
 *     the ray never left the widened box.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MAX_LAYERS 16
#define ORACLE_BOX_SLACK 1e-3

/* ------------------------------------------------------------------ */
/* networks                                                            */
/* ------------------------------------------------------------------ */

typedef struct {
    int in_dim, width, n_hidden;
    int n_sine;                        /* n_hidden + 1 sine layers (Eq. 2 f_0..f_{n-1}) */
    double omega0, omega;
    double *W[ORACLE_MAX_LAYERS];      /* folded sine-layer weights, row-major (out x in) */
    double *b[ORACLE_MAX_LAYERS];      /* folded sine-layer biases */
    double *w_out;                     /* linear output row W_n (width) */
    double b_out;                      /* b_n */
} oracle_net;

static uint32_t rd_u32(const unsigned char *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static float rd_f32(const unsigned char *p) {
    uint32_t u = rd_u32(p);
    float f;
    memcpy(&f, &u, 4);
    return f;
}

void oracle_net_free(oracle_net *n) {
    if (!n) return;
    for (int i = 0; i < ORACLE_MAX_LAYERS; ++i) {
        free(n->W[i]);
        free(n->b[i]);
    }
    free(n->w_out);
    free(n);
}

/* Parse an SDFN byte image.  Returns NULL on any format error. */
oracle_net *oracle_net_from_bytes(const unsigned char *buf, size_t len) {
    if (len < 32 || memcmp(buf, "SDFN", 4) != 0) return NULL;
    uint32_t version = rd_u32(buf + 4), in_dim = rd_u32(buf + 8), width = rd_u32(buf + 12);
    uint32_t n_hidden = rd_u32(buf + 16), flags = rd_u32(buf + 28);
    double omega0 = rd_f32(buf + 20), omega = rd_f32(buf + 24);
    if (version != 1 || in_dim < 1 || in_dim > 4 || width < 1 || width > 4096 ||
        n_hidden + 1 > ORACLE_MAX_LAYERS)
        return NULL;
    size_t count = (size_t)width * in_dim + width + (size_t)n_hidden * ((size_t)width * width + width) + width + 1;
    if (len != 32 + 4 * count) return NULL;
    int folded = (flags & 1u) != 0;

    oracle_net *n = (oracle_net *)calloc(1, sizeof(oracle_net));
    n->in_dim = (int)in_dim;
    n->width = (int)width;
    n->n_hidden = (int)n_hidden;
    n->n_sine = (int)n_hidden + 1;
    n->omega0 = omega0;
    n->omega = omega;
    const unsigned char *q = buf + 32;
    for (int l = 0; l < n->n_sine; ++l) {
        int fan_in = (l == 0) ? n->in_dim : n->width;
        double scale = folded ? 1.0 : (l == 0 ? omega0 : omega);
        n->W[l] = (double *)malloc(sizeof(double) * (size_t)width * fan_in);
        n->b[l] = (double *)malloc(sizeof(double) * width);
        for (size_t i = 0; i < (size_t)width * fan_in; ++i, q += 4) n->W[l][i] = scale * (double)rd_f32(q);
        for (size_t i = 0; i < width; ++i, q += 4) n->b[l][i] = scale * (double)rd_f32(q);
    }
    n->w_out = (double *)malloc(sizeof(double) * width);
    for (size_t i = 0; i < width; ++i, q += 4) n->w_out[i] = (double)rd_f32(q);
    n->b_out = (double)rd_f32(q);
    return n;
}

oracle_net *oracle_net_load(const char *path) {
    FILE *fp = fopen(path, "rb");
    if (!fp) return NULL;
    fseek(fp, 0, SEEK_END);
    long len = ftell(fp);
    fseek(fp, 0, SEEK_SET);
    if (len <= 0) {
        fclose(fp);
        return NULL;
    }
    unsigned char *buf = (unsigned char *)malloc((size_t)len);
    size_t got = fread(buf, 1, (size_t)len, fp);
    fclose(fp);
    oracle_net *n = (got == (size_t)len) ? oracle_net_from_bytes(buf, (size_t)len) : NULL;
    free(buf);
    return n;
}

void oracle_net_shape(const oracle_net *n, int *in_dim, int *width, int *n_hidden) {
    *in_dim = n->in_dim;
    *width = n->width;
    *n_hidden = n->n_hidden;
}

/* Eq. 2: f(p) = W_n f_{n-1}(...f_0(p)) + b_n with f_i(x) = sin(W_i x + b_i). */
double oracle_net_eval(const oracle_net *n, const double *p) {
    int w = n->width;
    double *x = (double *)malloc(sizeof(double) * w);
    double *y = (double *)malloc(sizeof(double) * w);
    for (int r = 0; r < w; ++r) {
        double a = n->b[0][r];
        for (int c = 0; c < n->in_dim; ++c) a += n->W[0][(size_t)r * n->in_dim + c] * p[c];
        x[r] = sin(a);
    }
    for (int l = 1; l < n->n_sine; ++l) {
        for (int r = 0; r < w; ++r) {
            double a = n->b[l][r];
            for (int c = 0; c < w; ++c) a += n->W[l][(size_t)r * w + c] * x[c];
            y[r] = sin(a);
        }
        double *t = x;
        x = y;
        y = t;
    }
    double f = n->b_out;
    for (int r = 0; r < w; ++r) f += n->w_out[r] * x[r];
    free(x);
    free(y);
    return f;
}

/* Alg. 2 for one point (k = 1 column of P), coordinate j = 0..in_dim-1 each in
 * its own loop exactly as written: the forward pass A_i is recomputed inside
 * every coordinate loop.
 *   input layer:  A_0 = W_0 p + b_0;  G_0 = W_0[:, j] (.) cos(A_0);  P_0 = sin(A_0)
 *   hidden i:     A_i = W_i P_{i-1} + b_i;  G_i = (W_i G_{i-1}) (.) cos(A_i);  P_i = sin(A_i)
 *   output:       grad_j = W_n G_{n-1}
 * The second form of G_i is the Hadamard identity of Sec. 5.1 applied to
 * Eq. 4, J f_i = W_i (.) cos[a_i | ... | a_i]. */
void oracle_net_grad(const oracle_net *n, const double *p, double *grad) {
    int w = n->width;
    double *A = (double *)malloc(sizeof(double) * w);
    double *P = (double *)malloc(sizeof(double) * w);
    double *G = (double *)malloc(sizeof(double) * w);
    double *P2 = (double *)malloc(sizeof(double) * w);
    double *G2 = (double *)malloc(sizeof(double) * w);
    for (int j = 0; j < n->in_dim; ++j) {
        for (int r = 0; r < w; ++r) {
            double a = n->b[0][r];
            for (int c = 0; c < n->in_dim; ++c) a += n->W[0][(size_t)r * n->in_dim + c] * p[c];
            A[r] = a;
        }
        for (int r = 0; r < w; ++r) {
            G[r] = n->W[0][(size_t)r * n->in_dim + j] * cos(A[r]);
            P[r] = sin(A[r]);
        }
        for (int l = 1; l < n->n_sine; ++l) {
            for (int r = 0; r < w; ++r) {
                double a = n->b[l][r], g = 0.0;
                for (int c = 0; c < w; ++c) {
                    a += n->W[l][(size_t)r * w + c] * P[c];
                    g += n->W[l][(size_t)r * w + c] * G[c];
                }
                A[r] = a;
                G2[r] = g;
            }
            for (int r = 0; r < w; ++r) {
                G2[r] *= cos(A[r]);
                P2[r] = sin(A[r]);
            }
            double *t = P;
            P = P2;
            P2 = t;
            t = G;
            G = G2;
            G2 = t;
        }
        double g = 0.0;
        for (int r = 0; r < w; ++r) g += n->w_out[r] * G[r];
        grad[j] = g;
    }
    free(A);
    free(P);
    free(G);
    free(P2);
    free(G2);
}

/* Largest singular value of an (rows x cols) matrix by power iteration on
 * M^T M, to relative change 1e-15 (at most 100000 iterations). */
static double spectral_norm(const double *M, int rows, int cols) {
    double *x = (double *)malloc(sizeof(double) * cols);
    double *y = (double *)malloc(sizeof(double) * rows);
    for (int c = 0; c < cols; ++c) x[c] = 1.0 + 0.001 * c;
    double sigma = 0.0;
    for (int it = 0; it < 100000; ++it) {
        double nx = 0.0;
        for (int c = 0; c < cols; ++c) nx += x[c] * x[c];
        nx = sqrt(nx);
        if (nx == 0.0) break;
        for (int c = 0; c < cols; ++c) x[c] /= nx;
        for (int r = 0; r < rows; ++r) {
            double s = 0.0;
            for (int c = 0; c < cols; ++c) s += M[(size_t)r * cols + c] * x[c];
            y[r] = s;
        }
        double ny = 0.0;
        for (int r = 0; r < rows; ++r) ny += y[r] * y[r];
        double s_new = sqrt(ny);
        for (int c = 0; c < cols; ++c) {
            double s = 0.0;
            for (int r = 0; r < rows; ++r) s += M[(size_t)r * cols + c] * y[r];
            x[c] = s;
        }
        if (it > 10 && fabs(s_new - sigma) <= 1e-15 * s_new) {
            sigma = s_new;
            break;
        }
        sigma = s_new;
    }
    free(x);
    free(y);
    return sigma;
}

/* Lipschitz bound of Eq. 2: sin is 1-Lipschitz, so L = prod_i ||W_i||_2 over
 * all sine layers (folded) times ||W_n||_2 of the output row. */
double oracle_lipschitz(const oracle_net *n) {
    double L = spectral_norm(n->W[0], n->width, n->in_dim);
    for (int l = 1; l < n->n_sine; ++l) L *= spectral_norm(n->W[l], n->width, n->width);
    double s = 0.0;
    for (int r = 0; r < n->width; ++r) s += n->w_out[r] * n->w_out[r];
    return L * sqrt(s);
}

/* ------------------------------------------------------------------ */
/* analytic SDFs used to pin the tracer                                */
/* ------------------------------------------------------------------ */

enum { SDF_KIND_NET = 0, SDF_KIND_SPHERE = 1, SDF_KIND_TORUS = 2 };

typedef struct {
    int kind;
    const oracle_net *net;   /* SDF_KIND_NET */
    double c[3], r, R;       /* sphere centre/radius; torus about the z axis: major R, minor r */
    double time;             /* 4th input of 4-D nets */
} oracle_sdf;

static double sdf_value(const oracle_sdf *s, const double *p) {
    switch (s->kind) {
    case SDF_KIND_NET: {
        if (s->net->in_dim == 4) {
            double q[4] = {p[0], p[1], p[2], s->time};
            return oracle_net_eval(s->net, q);
        }
        return oracle_net_eval(s->net, p);
    }
    case SDF_KIND_SPHERE: {
        double dx = p[0] - s->c[0], dy = p[1] - s->c[1], dz = p[2] - s->c[2];
        return sqrt(dx * dx + dy * dy + dz * dz) - s->r;
    }
    case SDF_KIND_TORUS: {
        double dx = p[0] - s->c[0], dy = p[1] - s->c[1], dz = p[2] - s->c[2];
        double q = sqrt(dx * dx + dy * dy) - s->R;
        return sqrt(q * q + dz * dz) - s->r;
    }
    }
    return NAN;
}

double oracle_sdf_value(const oracle_sdf *s, const double *p) { return sdf_value(s, p); }

/* ------------------------------------------------------------------ */
/* Alg. 1: multiscale sphere tracing                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    int n_levels;
    const oracle_sdf *levels;   /* f_1 .. f_m */
    const double *delta;        /* delta_j; delta_m used only when final_mode == 1 */
    const int *cap;             /* iteration cap per level */
    const double *scale;        /* step scale s_j */
    double eps;
    double box_lo, box_hi;
    int final_mode;             /* 0: trace S_m (Alg. 1); 1: stop on the delta_m shell of f_m */
} oracle_trace_params;

typedef struct {
    int hit;
    int iters;                  /* total steps over all levels */
    double p[3];
    double tau;                 /* distance travelled along the ray from its origin */
} oracle_ray_result;

static int outside_box(const double *p, double lo, double hi) {
    for (int c = 0; c < 3; ++c)
        if (p[c] < lo - ORACLE_BOX_SLACK || p[c] > hi + ORACLE_BOX_SLACK) return 1;
    return 0;
}

/* One ray.  If traj != NULL, up to traj_cap points (after each step) are
 * written there (3 doubles each) and their number is returned through
 * *traj_len; traj_level receives the level of each step. */
void oracle_trace_ray(const oracle_trace_params *P, const double *o, const double *v, oracle_ray_result *res,
                      double *traj, int *traj_level, int traj_cap, int *traj_len) {
    double tn = -INFINITY, tf = INFINITY;
    int missed = 0;
    for (int c = 0; c < 3; ++c) {
        if (v[c] != 0.0) {
            double t1 = (P->box_lo - o[c]) / v[c], t2 = (P->box_hi - o[c]) / v[c];
            double a = t1 < t2 ? t1 : t2, b = t1 < t2 ? t2 : t1;
            if (a > tn) tn = a;
            if (b < tf) tf = b;
        } else if (o[c] < P->box_lo || o[c] > P->box_hi) {
            missed = 1;
        }
    }
    if (tn < 0.0) tn = 0.0;
    if (traj_len) *traj_len = 0;
    res->hit = 0;
    res->iters = 0;
    if (missed || tn > tf) {
        res->p[0] = o[0];
        res->p[1] = o[1];
        res->p[2] = o[2];
        res->tau = 0.0;
        return;
    }
    double p[3] = {o[0] + tn * v[0], o[1] + tn * v[1], o[2] + tn * v[2]};
    double tau = tn;
    int total = 0, converged = 0;
    for (int j = 0; j < P->n_levels && !missed; ++j) {
        int last = (j == P->n_levels - 1);
        double d = (last && P->final_mode == 0) ? 0.0 : P->delta[j];
        double t = INFINITY;
        int k = 0;
        while (t > P->eps && k < P->cap[j]) {
            t = sdf_value(&P->levels[j], p) - d;
            double step = P->scale[j] * t;
            p[0] += step * v[0];
            p[1] += step * v[1];
            p[2] += step * v[2];
            tau += step;
            ++k;
            ++total;
            if (traj && traj_len && *traj_len < traj_cap) {
                memcpy(traj + 3 * (*traj_len), p, sizeof(p));
                if (traj_level) traj_level[*traj_len] = j;
                ++*traj_len;
            }
            if (outside_box(p, P->box_lo, P->box_hi)) {
                missed = 1;
                break;
            }
        }
        if (last) converged = (t <= P->eps);
    }
    res->hit = (!missed && converged) ? 1 : 0;
    res->iters = total;
    res->p[0] = p[0];
    res->p[1] = p[1];
    res->p[2] = p[2];
    res->tau = tau;
}

/* ------------------------------------------------------------------ */
/* dense march + bisection: the plain definition of the first hit      */
/* ------------------------------------------------------------------ */

/* First root of f along o + t v for t in [t0, t1]: march with step h until
 * the sign of f changes (or f == 0), then bisect to |interval| <= tol.
 * Returns 1 and *t_root on success, 0 if no sign change was found. */
int oracle_first_root(const oracle_sdf *s, const double *o, const double *v, double t0, double t1, double h,
                      double tol, double *t_root) {
    double p[3];
    double ta = t0;
    for (int c = 0; c < 3; ++c) p[c] = o[c] + ta * v[c];
    double fa = sdf_value(s, p);
    if (fa == 0.0) {
        *t_root = ta;
        return 1;
    }
    long nsteps = (long)ceil((t1 - t0) / h);
    for (long i = 1; i <= nsteps; ++i) {
        double tb = t0 + (double)i * h;
        if (tb > t1) tb = t1;
        for (int c = 0; c < 3; ++c) p[c] = o[c] + tb * v[c];
        double fb = sdf_value(s, p);
        if (fb == 0.0) {
            *t_root = tb;
            return 1;
        }
        if ((fa > 0) != (fb > 0)) {
            double lo = ta, hi = tb;
            while (hi - lo > tol) {
                double m = 0.5 * (lo + hi);
                for (int c = 0; c < 3; ++c) p[c] = o[c] + m * v[c];
                double fm = sdf_value(s, p);
                if ((fm > 0) == (fa > 0))
                    lo = m;
                else
                    hi = m;
            }
            *t_root = 0.5 * (lo + hi);
            return 1;
        }
        ta = tb;
        fa = fb;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* thresholds of Sec. 3.3                                              */
/* ------------------------------------------------------------------ */

/* Prop. 1: delta_m = e_m, delta_{i-1} = delta_i + e_i (i = m..2).
 * Arrays are 0-based: e[0] = varepsilon_1 ... e[m-1] = varepsilon_m. */
void oracle_thresholds_prop1(const double *e, int m, double *delta) {
    delta[m - 1] = e[m - 1];
    for (int i = m - 1; i >= 1; --i) delta[i - 1] = delta[i] + e[i];
}

/* Prop. 2: delta_m = e_m + e_{m-1}, delta_{i-1} = delta_i + e_i + e_{i-1}. */
void oracle_thresholds_prop2(const double *e, int m, double *delta) {
    delta[m - 1] = e[m - 1] + (m >= 2 ? e[m - 2] : 0.0);
    for (int i = m - 1; i >= 1; --i) delta[i - 1] = delta[i] + e[i] + e[i - 1];
}

/* ------------------------------------------------------------------ */
/* batched drivers (threads over rays / points)                        */
/* ------------------------------------------------------------------ */

typedef struct {
    const oracle_trace_params *P;
    const float *orig, *dir;   /* SoA (3, n) float32 */
    const int64_t *idx;        /* optional subset of ray indices */
    int64_t n, stride;
    int64_t begin, end;
    float *out_pos, *out_tau;  /* SoA (3, n) / (n) over the processed list */
    uint8_t *out_hit;
    int32_t *out_iters;
    double *out_pos64;         /* optional (3, n) float64 */
} trace_job;

static void *trace_worker(void *arg) {
    trace_job *J = (trace_job *)arg;
    for (int64_t k = J->begin; k < J->end; ++k) {
        int64_t i = J->idx ? J->idx[k] : k;
        double o[3] = {J->orig[i], J->orig[J->stride + i], J->orig[2 * J->stride + i]};
        double v[3] = {J->dir[i], J->dir[J->stride + i], J->dir[2 * J->stride + i]};
        oracle_ray_result r;
        oracle_trace_ray(J->P, o, v, &r, NULL, NULL, 0, NULL);
        for (int c = 0; c < 3; ++c) {
            if (J->out_pos) J->out_pos[c * J->n + k] = (float)r.p[c];
            if (J->out_pos64) J->out_pos64[c * J->n + k] = r.p[c];
        }
        if (J->out_tau) J->out_tau[k] = (float)r.tau;
        if (J->out_hit) J->out_hit[k] = (uint8_t)r.hit;
        if (J->out_iters) J->out_iters[k] = r.iters;
    }
    return NULL;
}

/* Trace rays idx[0..n) (or 0..n when idx == NULL) of the SoA arrays with row
 * stride `stride`; results are written densely in list order. */
int oracle_trace_batch(const oracle_trace_params *P, const float *orig, const float *dir, int64_t stride,
                       const int64_t *idx, int64_t n, float *out_pos, double *out_pos64, float *out_tau,
                       uint8_t *out_hit, int32_t *out_iters, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    pthread_t th[512];
    trace_job jobs[512];
    int64_t chunk = (n + n_threads - 1) / n_threads;
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        trace_job *J = &jobs[t];
        J->P = P;
        J->orig = orig;
        J->dir = dir;
        J->idx = idx;
        J->n = n;
        J->stride = stride;
        J->begin = t * chunk;
        J->end = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        J->out_pos = out_pos;
        J->out_pos64 = out_pos64;
        J->out_tau = out_tau;
        J->out_hit = out_hit;
        J->out_iters = out_iters;
        if (J->begin >= J->end) break;
        pthread_create(&th[t], NULL, trace_worker, J);
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return 0;
}

typedef struct {
    const oracle_net *net;
    const double *pts;   /* SoA (in_dim or 3, stride) float64 */
    int64_t stride, n, begin, end;
    double time;
    double *out_grad;    /* SoA (3, n) */
    double *out_val;     /* (n) or NULL */
} grad_job;

static void *grad_worker(void *arg) {
    grad_job *J = (grad_job *)arg;
    for (int64_t k = J->begin; k < J->end; ++k) {
        double p[4] = {J->pts[k], J->pts[J->stride + k], J->pts[2 * J->stride + k], J->time};
        double g[4];
        oracle_net_grad(J->net, p, g);
        for (int c = 0; c < 3; ++c) J->out_grad[c * J->n + k] = g[c];
        if (J->out_val) J->out_val[k] = oracle_net_eval(J->net, p);
    }
    return NULL;
}

/* Alg. 2 over n points (SoA float64 (3, n)); also f(p) when out_val != NULL. */
int oracle_grad_batch(const oracle_net *net, const double *pts, int64_t n, double time, double *out_grad,
                      double *out_val, int n_threads) {
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    pthread_t th[512];
    grad_job jobs[512];
    int64_t chunk = (n + n_threads - 1) / n_threads;
    int started = 0;
    for (int t = 0; t < n_threads; ++t) {
        grad_job *J = &jobs[t];
        J->net = net;
        J->pts = pts;
        J->stride = n;
        J->n = n;
        J->time = time;
        J->begin = t * chunk;
        J->end = (t + 1) * chunk < n ? (t + 1) * chunk : n;
        J->out_grad = out_grad;
        J->out_val = out_val;
        if (J->begin >= J->end) break;
        pthread_create(&th[t], NULL, grad_worker, J);
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* Sec. 5 neural normal mapping: N(p) = grad f(p) / |grad f(p)| at every
 * point with mask != 0; (0, 0, 0) where masked out or |grad f| < 1e-12. */
int oracle_normal_map(const oracle_net *net, const double *pts, const uint8_t *mask, int64_t n, double time,
                      double *out_normal, int n_threads) {
    oracle_grad_batch(net, pts, n, time, out_normal, NULL, n_threads);
    for (int64_t k = 0; k < n; ++k) {
        double g[3] = {out_normal[k], out_normal[n + k], out_normal[2 * n + k]};
        double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
        int keep = (!mask || mask[k]) && len >= 1e-12;
        for (int c = 0; c < 3; ++c) out_normal[c * n + k] = keep ? g[c] / len : 0.0;
    }
    return 0;
}
