/*
 * acpr_oracle.c -- plain, slow, float64 CPU oracle for the Parareal / Allen-Cahn
 * hot path.  TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU
 * baseline leg of the benchmark call it; the library never does.  It shares no
 * code with the CUDA path.
 *
 * Every routine follows the paper's definitions in their stated order, with no
 * blocking or fusion:
 *   - Allen-Cahn models and double-well nonlinearity f(u) = u - u^3: Sec. 2,
 *     Eq. (class_AC_eq) and Eq. (mass_AC_eq).
 *   - Energy E(u) = int eps^2/2 |grad u|^2 + F(u): Sec. 2, Eq. (energy).
 *   - Grid: N unknowns per side, h = L/N, x_i = -L/2 + i h (Sec. 3.1, periodic
 *     identification U^0 = U^N).
 *   - Fine step: stabilised linear semi-implicit scheme with the periodic
 *     5-point Laplacian, solved by the 2D DFT (the scheme family the paper cites
 *     in Sec. 1; the spatial options are in Sec. 3.1).
 *   - Crank-Nicolson fine step with Picard iteration (the paper's own fine
 *     scheme, Sec. 3.1, Eq. (fully-discrete)): or_cn_step, or_cn_propagate.
 *   - Coarse propagator: 3x3 circular-padded conv stack (Sec. 3.2); the
 *     paper's ResBlock ACNN / mACNN, its scheme-residual loss (Eq. loss_ACN),
 *     Adam and the training loop of Algorithm 1 (Sec. 3.2).
 *   - Parareal: Algorithm 2 / Sec. 3.3, with G composed m times per slice (the
 *     remark after Algorithm 2).
 *   - The fine step, the ResBlock ACNN (3x3x3) and Algorithm 2 on the periodic
 *     cube (the 3D experiments of Sec. 4).
 *
 * Threads: or_set_threads(t) lets conv3x3 split its output rows, and
 * Algorithm 2 its independent fine solves, over t POSIX threads.  Each output
 * value is computed by exactly the same loop as with one thread, so results
 * do not depend on t (this only shortens the wall time of large cases).
 *
 * Parity status: every function here is pinned by the not-gpu tests (naive DFT,
 * dense linear solve, closed forms, invariants, finite differences, brute force,
 * library routines).  The straight-through backward of the bf16-emulating conv
 * mode is pinned as the exact gradient (central differences) of the stack with
 * each rounding frozen into a constant offset at the evaluation point.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int n;          /* grid points per side */
    double length;  /* side of the periodic square */
    double eps;     /* interface width epsilon */
    double S;       /* stabilisation constant */
    double dt;      /* fine time step */
    int variant;    /* 0 classic, 1 mass-conserving */
} or_params;

typedef struct {
    int layers;     /* number of 3x3 convolutions */
    int channels;   /* hidden width C */
    int act;        /* 0 tanh, 1 gelu (erf form) */
    int residual;   /* 1: output = input + stack(input) */
    int mass_fix;   /* 1: add mean(input) - mean(output) to every entry */
    int limiter;    /* 1: clamp to [lo, hi] */
    int bf16;       /* 1: round weights, conv input and hidden activations to bf16 */
    double lo, hi;
    const double* w; /* concat over layers of W_l[cout][cin][3][3] */
    const double* b; /* concat over layers of b_l[cout] */
} or_cnn;

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------ threads ---- */
static int g_threads = 1;

void or_set_threads(int t) { g_threads = t < 1 ? 1 : (t > 256 ? 256 : t); }
int or_get_threads(void) { return g_threads; }

typedef struct {
    void (*fn)(void* ctx, long lo, long hi);
    void* ctx;
    long lo, hi;
} or_task;

static void* or_task_run(void* a) {
    or_task* t = (or_task*)a;
    t->fn(t->ctx, t->lo, t->hi);
    return NULL;
}

/* Run fn(ctx, lo, hi) over [0, count) split into g_threads contiguous ranges. */
static void or_parallel_for(long count, void (*fn)(void*, long, long), void* ctx) {
    int t = g_threads;
    if (t > count) t = (int)count;
    if (t <= 1) { if (count > 0) fn(ctx, 0, count); return; }
    pthread_t th[256];
    or_task task[256];
    int started[256];
    for (int i = 0; i < t; i++) {
        task[i].fn = fn; task[i].ctx = ctx;
        task[i].lo = count * i / t; task[i].hi = count * (i + 1) / t;
        started[i] = pthread_create(&th[i], NULL, or_task_run, &task[i]) == 0;
        if (!started[i]) or_task_run(&task[i]);
    }
    for (int i = 0; i < t; i++)
        if (started[i]) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------ FFT -- */
/* Recursive radix-2 decimation-in-time Cooley-Tukey transform,
 * y_k = sum_j x_j exp(sign * 2 pi i j k / n), unnormalised. */
static void fft_rec(const cplx* in, cplx* out, int n, int stride, int sign) {
    if (n == 1) { out[0] = in[0]; return; }
    int h = n / 2;
    fft_rec(in, out, h, 2 * stride, sign);
    fft_rec(in + stride, out + h, h, 2 * stride, sign);
    for (int k = 0; k < h; k++) {
        double ang = sign * 2.0 * PI * (double)k / (double)n;
        cplx w = cos(ang) + I * sin(ang);
        cplx e = out[k], o = w * out[k + h];
        out[k] = e + o;
        out[k + h] = e - o;
    }
}

void or_fft1d(cplx* x, int n, int sign) {
    cplx* in = malloc(sizeof(cplx) * n);
    memcpy(in, x, sizeof(cplx) * n);
    fft_rec(in, x, n, 1, sign);
    free(in);
}

/* 2D transform of a row-major n x n array: every row, then every column. */
void or_fft2d(cplx* x, int n, int sign) {
    cplx* col = malloc(sizeof(cplx) * n);
    for (int i = 0; i < n; i++) or_fft1d(x + (size_t)i * n, n, sign);
    for (int j = 0; j < n; j++) {
        for (int i = 0; i < n; i++) col[i] = x[(size_t)i * n + j];
        or_fft1d(col, n, sign);
        for (int i = 0; i < n; i++) x[(size_t)i * n + j] = col[i];
    }
    free(col);
}

/* Direct O(n^4) 2D DFT, the definition itself. */
void or_dft2d_naive(const cplx* x, cplx* y, int n, int sign) {
    for (int k = 0; k < n; k++)
        for (int l = 0; l < n; l++) {
            cplx acc = 0;
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    double ang = sign * 2.0 * PI * (double)(((long)i * k + (long)j * l) % n) / n;
                    acc += x[(size_t)i * n + j] * (cos(ang) + I * sin(ang));
                }
            y[(size_t)k * n + l] = acc;
        }
}

/* Interleaved (re, im) wrappers for callers without C99 complex. */
void or_fft2d_ri(double* xri, int n, int sign) { or_fft2d((cplx*)xri, n, sign); }
void or_dft2d_naive_ri(const double* xri, double* yri, int n, int sign) {
    or_dft2d_naive((const cplx*)xri, (cplx*)yri, n, sign);
}

/* ------------------------------------------------------------- model ---- */
static double f_dw(double u) { return u - u * u * u; }          /* f = -F' */
static double fprime_dw(double u) { return 1.0 - 3.0 * u * u; }
static double F_dw(double u) { double t = u * u - 1.0; return 0.25 * t * t; }

/* Eigenvalue of the periodic 5-point Laplacian for mode (k, l):
 * -(4/h^2) (sin^2(pi k/N) + sin^2(pi l/N)). */
static double lap_symbol(int k, int l, int n, double h) {
    double sk = sin(PI * k / n), sl = sin(PI * l / n);
    return -(4.0 / (h * h)) * (sk * sk + sl * sl);
}

/* Solve ((1 + S dt) I - dt eps^2 Lap_h) v = r by the 2D DFT. */
static void solve_A(const or_params* p, const double* r, double* v) {
    int n = p->n;
    double h = p->length / n;
    cplx* z = malloc(sizeof(cplx) * n * n);
    for (int i = 0; i < n * n; i++) z[i] = r[i];
    or_fft2d(z, n, -1);
    for (int k = 0; k < n; k++)
        for (int l = 0; l < n; l++) {
            double D = 1.0 + p->S * p->dt - p->dt * p->eps * p->eps * lap_symbol(k, l, n, h);
            z[(size_t)k * n + l] /= D;
        }
    or_fft2d(z, n, +1);
    for (int i = 0; i < n * n; i++) v[i] = creal(z[i]) / ((double)n * n);
    free(z);
}

void or_solve_A(const or_params* p, const double* r, double* v) { solve_A(p, r, v); }

/* One stabilised semi-implicit step:
 *   (1 + S dt) u' - dt eps^2 Lap_h u' = (1 + S dt) u + dt (f(u) - beta),
 * beta = 0 (classic) or beta = mean_x f(u) (mass-conserving Lagrange multiplier,
 * Eq. (mass_AC_eq) evaluated explicitly at u^n). */
void or_fine_step(const or_params* p, const double* u, double* out) {
    int n = p->n, m = n * n;
    double beta = 0.0;
    if (p->variant == 1) {
        for (int i = 0; i < m; i++) beta += f_dw(u[i]);
        beta /= m;
    }
    double* r = malloc(sizeof(double) * m);
    for (int i = 0; i < m; i++) r[i] = (1.0 + p->S * p->dt) * u[i] + p->dt * (f_dw(u[i]) - beta);
    solve_A(p, r, out);
    free(r);
}

/* Fine propagator over one slice: `steps` fine steps. */
void or_fine_propagate(const or_params* p, int steps, const double* u, double* out) {
    int m = p->n * p->n;
    double* a = malloc(sizeof(double) * m);
    memcpy(a, u, sizeof(double) * m);
    for (int s = 0; s < steps; s++) {
        or_fine_step(p, a, out);
        memcpy(a, out, sizeof(double) * m);
    }
    if (steps == 0) memcpy(out, u, sizeof(double) * m);
    free(a);
}

/* 5-point periodic Laplacian applied directly (defined below). */
static void apply_lap(int n, double h, const double* u, double* out);

/* Solve (I - dt/2 eps^2 Lap_h) v = r by the 2D DFT (the linear system of each
 * Picard iteration in Sec. 3.1). */
static void solve_cn(const or_params* p, const double* r, double* v) {
    int n = p->n;
    double h = p->length / n;
    cplx* z = malloc(sizeof(cplx) * n * n);
    for (int i = 0; i < n * n; i++) z[i] = r[i];
    or_fft2d(z, n, -1);
    for (int k = 0; k < n; k++)
        for (int l = 0; l < n; l++) {
            double D = 1.0 - 0.5 * p->dt * p->eps * p->eps * lap_symbol(k, l, n, h);
            z[(size_t)k * n + l] /= D;
        }
    or_fft2d(z, n, +1);
    for (int i = 0; i < n * n; i++) v[i] = creal(z[i]) / ((double)n * n);
    free(z);
}

/* One Crank-Nicolson step of Sec. 3.1,
 *   (U' - U)/dt = eps^2 Lap_h (U' + U)/2 + (f(U') + f(U))/2 - g(U, U'),
 * g = 0 (classic) or g = mean_x (f(U') + f(U))/2 (mass-conserving), solved by
 * the Picard iteration of Sec. 3.1: U^0 = U and
 *   (I - dt/2 eps^2 Lap_h) U^{m+1} = U + dt/2 eps^2 Lap_h U + dt/2 (f(U) + f(U^m)) - dt g(U, U^m)
 * until max |U^{m+1} - U^m| <= tol or maxit iterations; U' = the last iterate.
 * (The rearranged Eq. (fully-discrete) prints dt/2 g; the first form, whose
 * mean of the right-hand side vanishes, gives dt g, used here.)  Returns the
 * number of iterations. */
int or_cn_step(const or_params* p, const double* u, double* out, double tol, int maxit) {
    int n = p->n, m = n * n;
    double h = p->length / n;
    double* r0 = malloc(sizeof(double) * m);
    double* r = malloc(sizeof(double) * m);
    double* um = malloc(sizeof(double) * m);
    double* lap = malloc(sizeof(double) * m);
    apply_lap(n, h, u, lap);
    for (int i = 0; i < m; i++) r0[i] = u[i] + 0.5 * p->dt * (p->eps * p->eps * lap[i] + f_dw(u[i]));
    memcpy(um, u, sizeof(double) * m);
    int it = 0;
    while (it < maxit) {
        double g = 0.0;
        if (p->variant == 1) {
            for (int i = 0; i < m; i++) g += 0.5 * (f_dw(um[i]) + f_dw(u[i]));
            g /= m;
        }
        for (int i = 0; i < m; i++) r[i] = r0[i] + 0.5 * p->dt * f_dw(um[i]) - p->dt * g;
        solve_cn(p, r, out);
        ++it;
        double diff = 0.0;
        for (int i = 0; i < m; i++) {
            double d = fabs(out[i] - um[i]);
            if (d > diff) diff = d;
        }
        memcpy(um, out, sizeof(double) * m);
        if (diff <= tol) break;
    }
    if (it == 0) memcpy(out, u, sizeof(double) * m);
    free(r0);
    free(r);
    free(um);
    free(lap);
    return it;
}

/* `steps` Crank-Nicolson steps; returns the total number of Picard iterations. */
long or_cn_propagate(const or_params* p, int steps, const double* u, double* out, double tol, int maxit) {
    int m = p->n * p->n;
    double* a = malloc(sizeof(double) * m);
    memcpy(a, u, sizeof(double) * m);
    long total = 0;
    for (int s = 0; s < steps; s++) {
        total += or_cn_step(p, a, out, tol, maxit);
        memcpy(a, out, sizeof(double) * m);
    }
    if (steps == 0) memcpy(out, u, sizeof(double) * m);
    free(a);
    return total;
}

/* Discrete energy E_h(u) = h^2 sum eps^2/2 (|D+x u|^2 + |D+y u|^2) + F(u). */
double or_energy(const or_params* p, const double* u) {
    int n = p->n;
    double h = p->length / n, e = 0.0;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) {
            double c = u[i * n + j];
            double dx = (u[((i + 1) % n) * n + j] - c) / h;
            double dy = (u[i * n + (j + 1) % n] - c) / h;
            e += 0.5 * p->eps * p->eps * (dx * dx + dy * dy) + F_dw(c);
        }
    return h * h * e;
}

/* Mass M = h^2 sum u. */
double or_mass(const or_params* p, const double* u) {
    double h = p->length / p->n, s = 0.0;
    for (int i = 0; i < p->n * p->n; i++) s += u[i];
    return h * h * s;
}

/* 5-point periodic Laplacian applied directly (used by the energy gradient). */
static void apply_lap(int n, double h, const double* u, double* out) {
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            out[i * n + j] = (u[((i + 1) % n) * n + j] + u[((i + n - 1) % n) * n + j] +
                              u[i * n + (j + 1) % n] + u[i * n + (j + n - 1) % n] -
                              4.0 * u[i * n + j]) / (h * h);
}

/* dE_h/du = h^2 (-eps^2 Lap_h u - f(u)). */
void or_energy_grad(const or_params* p, const double* u, double* g) {
    int n = p->n, m = n * n;
    double h = p->length / n;
    double* lu = malloc(sizeof(double) * m);
    apply_lap(n, h, u, lu);
    for (int i = 0; i < m; i++) g[i] = h * h * (-p->eps * p->eps * lu[i] - f_dw(u[i]));
    free(lu);
}

/* Transposed Jacobian of one fine step at u^n applied to lam (the adjoint step):
 * u' = A^{-1} ((1+S dt) u + dt (f(u) - beta(u))), A symmetric, so with
 * mu = A^{-1} lam:  lam_n = (1+S dt) mu + dt f'(u) * (mu - [mass] mean(mu)). */
void or_fine_adjoint_step(const or_params* p, const double* u, const double* lam, double* out) {
    int m = p->n * p->n;
    double* mu = malloc(sizeof(double) * m);
    solve_A(p, lam, mu);
    double mbar = 0.0;
    if (p->variant == 1) {
        for (int i = 0; i < m; i++) mbar += mu[i];
        mbar /= m;
    }
    for (int i = 0; i < m; i++)
        out[i] = (1.0 + p->S * p->dt) * mu[i] + p->dt * fprime_dw(u[i]) * (mu[i] - mbar);
    free(mu);
}

/* Gradient of E_h(u^steps) with respect to u^0 by storing every state and
 * running the adjoint steps backwards (no checkpointing: the plain form). */
void or_energy_gradient_through_solve(const or_params* p, int steps, const double* u0, double* grad) {
    int m = p->n * p->n;
    double* traj = malloc(sizeof(double) * (size_t)m * (steps + 1));
    memcpy(traj, u0, sizeof(double) * m);
    for (int s = 0; s < steps; s++) or_fine_step(p, traj + (size_t)s * m, traj + (size_t)(s + 1) * m);
    double* lam = malloc(sizeof(double) * m);
    double* tmp = malloc(sizeof(double) * m);
    or_energy_grad(p, traj + (size_t)steps * m, lam);
    for (int s = steps - 1; s >= 0; s--) {
        or_fine_adjoint_step(p, traj + (size_t)s * m, lam, tmp);
        memcpy(lam, tmp, sizeof(double) * m);
    }
    memcpy(grad, lam, sizeof(double) * m);
    free(traj); free(lam); free(tmp);
}

/* --------------------------------------------------------------- CNN ---- */
/* Round a double to the nearest bfloat16 value (ties to even). */
double or_round_bf16(double x) {
    if (!isfinite(x) || x == 0.0) return x;
    int e;
    double mant = frexp(fabs(x), &e);         /* |x| = mant * 2^e, mant in [0.5,1) */
    /* bf16 keeps 8 significant bits: scale so that the kept bits are integral */
    double scaled = ldexp(mant, 8);            /* in [128, 256) */
    double r = nearbyint(scaled);              /* ties to even under the default mode */
    double y = ldexp(r, e - 8);
    return x < 0 ? -y : y;
}

static double act_fn(int act, double x) {
    if (act == 0) return tanh(x);
    return 0.5 * x * (1.0 + erf(x / sqrt(2.0)));
}

static double act_grad(int act, double x) {
    if (act == 0) { double t = tanh(x); return 1.0 - t * t; }
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * exp(-0.5 * x * x) / sqrt(2.0 * PI);
}

/* One 3x3 cross-correlation with circular padding 1:
 * out[o][i][j] = b[o] + sum_{c,a,e} W[o][c][a][e] in[c][(i+a-1) mod n][(j+e-1) mod n]. */
typedef struct { int n, cin, cout; const double *W, *b, *in; double* out; } conv3x3_ctx;

/* Output rows r = o * n + i in [lo, hi). */
static void conv3x3_rows(void* vc, long lo, long hi) {
    const conv3x3_ctx* q = (const conv3x3_ctx*)vc;
    const int n = q->n, cin = q->cin;
    for (long r = lo; r < hi; r++) {
        const int o = (int)(r / n), i = (int)(r % n);
        for (int j = 0; j < n; j++) {
            double acc = q->b[o];
            for (int c = 0; c < cin; c++)
                for (int a = 0; a < 3; a++)
                    for (int e = 0; e < 3; e++) {
                        int ii = (i + a - 1 + n) % n, jj = (j + e - 1 + n) % n;
                        acc += q->W[((o * cin + c) * 3 + a) * 3 + e] * q->in[((size_t)c * n + ii) * n + jj];
                    }
            q->out[((size_t)o * n + i) * n + j] = acc;
        }
    }
}

static void conv3x3(int n, int cin, int cout, const double* W, const double* b,
                    const double* in, double* out) {
    conv3x3_ctx q = {n, cin, cout, W, b, in, out};
    or_parallel_for((long)cout * n, conv3x3_rows, &q);
}

static void layer_dims(const or_cnn* d, int l, int* cin, int* cout) {
    *cin = (l == 0) ? 1 : d->channels;
    *cout = (l == d->layers - 1) ? 1 : d->channels;
}

/* Forward pass.  If pre_acts != NULL, stores every layer's pre-activation
 * (z_l, [cout][n][n]) and post-activation input (a_l) for the backward pass;
 * the buffers are laid out layer after layer, C*n*n doubles per layer. */
static void cnn_forward_impl(const or_cnn* d, int n, const double* u, double* out,
                             double* pre_acts, double* inputs) {
    size_t m = (size_t)n * n;
    int C = d->channels > 1 ? d->channels : 1;
    double* a = malloc(sizeof(double) * C * m);
    double* z = malloc(sizeof(double) * C * m);
    for (size_t i = 0; i < m; i++) a[i] = d->bf16 ? or_round_bf16(u[i]) : u[i];
    const double* W = d->w;
    const double* B = d->b;
    int nw_total = 0, nb_total = 0;
    for (int l = 0; l < d->layers; l++) { int ci, co; layer_dims(d, l, &ci, &co); nw_total += ci * co * 9; nb_total += co; }
    double* wr = malloc(sizeof(double) * nw_total);
    for (int i = 0; i < nw_total; i++) wr[i] = d->bf16 ? or_round_bf16(W[i]) : W[i];
    int woff = 0, boff = 0;
    for (int l = 0; l < d->layers; l++) {
        int cin, cout;
        layer_dims(d, l, &cin, &cout);
        if (inputs) memcpy(inputs + (size_t)l * C * m, a, sizeof(double) * cin * m);
        conv3x3(n, cin, cout, wr + woff, B + boff, a, z);
        if (pre_acts) memcpy(pre_acts + (size_t)l * C * m, z, sizeof(double) * cout * m);
        woff += cin * cout * 9;
        boff += cout;
        if (l < d->layers - 1) {
            for (size_t i = 0; i < (size_t)cout * m; i++) {
                double v = act_fn(d->act, z[i]);
                a[i] = d->bf16 ? or_round_bf16(v) : v;
            }
        }
    }
    /* z holds the last layer's output (one channel) */
    for (size_t i = 0; i < m; i++) out[i] = d->residual ? u[i] + z[i] : z[i];
    if (d->mass_fix) {
        double mi = 0.0, mo = 0.0;
        for (size_t i = 0; i < m; i++) { mi += u[i]; mo += out[i]; }
        double shift = (mi - mo) / (double)m;
        for (size_t i = 0; i < m; i++) out[i] += shift;
    }
    if (d->limiter)
        for (size_t i = 0; i < m; i++) out[i] = out[i] < d->lo ? d->lo : (out[i] > d->hi ? d->hi : out[i]);
    free(a); free(z); free(wr);
}

void or_cnn_forward(const or_cnn* d, int n, const double* u, double* out) {
    cnn_forward_impl(d, n, u, out, NULL, NULL);
}

void or_cnn_forward_batch(const or_cnn* d, int n, int batch, const double* u, double* out) {
    for (int b = 0; b < batch; b++)
        cnn_forward_impl(d, n, u + (size_t)b * n * n, out + (size_t)b * n * n, NULL, NULL);
}

/* Backward pass of the residual stack without limiter: given dL/dout,
 * returns dL/du, dL/dW, dL/db (accumulated into gw, gb, which the caller
 * zeroes).  With the mACNN mass shift, out = u + s(u) - mean(s(u)), so the
 * stack receives dL/dout minus its mean.  With bf16 set, the products use the
 * same rounded weights and layer inputs as the forward pass (rounding is
 * passed through as the identity, the straight-through reading of the bf16
 * policy). */
void or_cnn_backward(const or_cnn* d, int n, const double* u, const double* gout,
                     double* gin, double* gw, double* gb) {
    size_t m = (size_t)n * n;
    int C = d->channels > 1 ? d->channels : 1;
    int L = d->layers;
    double* pre = malloc(sizeof(double) * (size_t)L * C * m);
    double* ins = malloc(sizeof(double) * (size_t)L * C * m);
    double* out = malloc(sizeof(double) * m);
    cnn_forward_impl(d, n, u, out, pre, ins);
    int* woffs = malloc(sizeof(int) * L);
    int* boffs = malloc(sizeof(int) * L);
    int woff = 0, boff = 0;
    for (int l = 0; l < L; l++) {
        int ci, co; layer_dims(d, l, &ci, &co);
        woffs[l] = woff; boffs[l] = boff; woff += ci * co * 9; boff += co;
    }
    int nw_total = woff;
    double* wr = malloc(sizeof(double) * (nw_total > 0 ? nw_total : 1));
    for (int i = 0; i < nw_total; i++) wr[i] = d->bf16 ? or_round_bf16(d->w[i]) : d->w[i];
    double* gz = malloc(sizeof(double) * C * m);   /* dL/dz_l */
    double* ga = malloc(sizeof(double) * C * m);   /* dL/da_l (layer input) */
    memcpy(gz, gout, sizeof(double) * m);          /* last layer: out = u + z_L */
    if (d->mass_fix) {
        double gm = 0.0;
        for (size_t i = 0; i < m; i++) gm += gout[i];
        gm /= (double)m;
        for (size_t i = 0; i < m; i++) gz[i] = gout[i] - gm;
    }
    for (int l = L - 1; l >= 0; l--) {
        int cin, cout;
        layer_dims(d, l, &cin, &cout);
        const double* W = wr + woffs[l];
        const double* a = ins + (size_t)l * C * m;
        /* db, dW */
        for (int o = 0; o < cout; o++)
            for (size_t i = 0; i < m; i++) gb[boffs[l] + o] += gz[(size_t)o * m + i];
        for (int o = 0; o < cout; o++)
            for (int c = 0; c < cin; c++)
                for (int aa = 0; aa < 3; aa++)
                    for (int e = 0; e < 3; e++) {
                        double acc = 0.0;
                        for (int i = 0; i < n; i++)
                            for (int j = 0; j < n; j++) {
                                int ii = (i + aa - 1 + n) % n, jj = (j + e - 1 + n) % n;
                                acc += gz[((size_t)o * n + i) * n + j] * a[((size_t)c * n + ii) * n + jj];
                            }
                        gw[woffs[l] + ((o * cin + c) * 3 + aa) * 3 + e] += acc;
                    }
        /* d input: scatter each output gradient back through the stencil */
        memset(ga, 0, sizeof(double) * cin * m);
        for (int o = 0; o < cout; o++)
            for (int i = 0; i < n; i++)
                for (int j = 0; j < n; j++) {
                    double g = gz[((size_t)o * n + i) * n + j];
                    for (int c = 0; c < cin; c++)
                        for (int aa = 0; aa < 3; aa++)
                            for (int e = 0; e < 3; e++) {
                                int ii = (i + aa - 1 + n) % n, jj = (j + e - 1 + n) % n;
                                ga[((size_t)c * n + ii) * n + jj] += W[((o * cin + c) * 3 + aa) * 3 + e] * g;
                            }
                }
        if (l > 0) {
            const double* zprev = pre + (size_t)(l - 1) * C * m;
            for (size_t i = 0; i < (size_t)cin * m; i++) gz[i] = ga[i] * act_grad(d->act, zprev[i]);
        }
    }
    for (size_t i = 0; i < m; i++) gin[i] = gout[i] + ga[i];   /* residual skip + stack */
    free(pre); free(ins); free(out); free(woffs); free(boffs); free(gz); free(ga); free(wr);
}

/* ---------------------------------------------------------- Parareal ---- */
/* Relative L2 and sup-norm increments between two trajectories over slices
 * j = 1..s (Sec. 3.3 convergence test; relative L2 reading of the tolerance). */
static void or_residual_len(int s, size_t m, const double* Unew, const double* Uold, double* l2, double* mx);

void or_residual(int s, int n, const double* Unew, const double* Uold, double* l2, double* mx) {
    or_residual_len(s, (size_t)n * n, Unew, Uold, l2, mx);
}

/* The same over slices of m values each (any dimension). */
static void or_residual_len(int s, size_t m, const double* Unew, const double* Uold, double* l2, double* mx) {
    double num = 0.0, den = 0.0, mxv = 0.0;
    for (int j = 1; j <= s; j++)
        for (size_t i = 0; i < m; i++) {
            double a = Unew[(size_t)j * m + i], d = a - Uold[(size_t)j * m + i];
            num += d * d;
            den += a * a;
            if (fabs(d) > mxv) mxv = fabs(d);
        }
    *l2 = den > 0 ? sqrt(num) / sqrt(den) : sqrt(num);
    *mx = mxv;
}

/* Algorithm 2.  U: [s+1][n][n] output trajectory (the last iterate).
 * res_l2 / res_max: per-iteration increments (index k = 1..); iters: the k at
 * which the loop stopped.  If coarse == NULL, G is the fine propagator itself
 * with `coarse_steps` fine steps (for the G = F property).  Returns the number
 * of coarse-propagator evaluations (the cost-model count of Sec. 3.4: the
 * stored G(U^{k-1}_n) values are reused, and U^k_{k-1} = U^{k-1}_{k-1} makes its
 * G value known).  G is re-evaluated literally as Algorithm 2 states it only
 * when `literal` is set. */
typedef struct or_acnn_s or_acnn;
void or_acnn_forward(const or_acnn* d, int n, int batch, const double* u, double* out);
void or_acnn3d_forward(const or_acnn* d, int n, int batch, const double* u, double* out);
void or_fine3d_propagate(const or_params* p, int steps, const double* u, double* out);

/* The coarse propagator of one solve: the conv stack, the ResBlock ACNN, or
 * (both NULL) F over coarse_steps fine steps; dim 2 (the square) or 3 (the
 * cube: the ACNN with 3 x 3 x 3 convolutions, or the 3D fine step). */
typedef struct { const or_cnn* cnn; const or_acnn* acnn; int coarse_steps; int dim; } or_coarse;

static size_t or_field_len(const or_params* p, int dim) {
    return dim == 3 ? (size_t)p->n * p->n * p->n : (size_t)p->n * p->n;
}

static void or_fine_any(const or_params* p, int dim, int steps, const double* in, double* out) {
    if (dim == 3) or_fine3d_propagate(p, steps, in, out);
    else or_fine_propagate(p, steps, in, out);
}

/* One application of the coarse propagator. */
static void or_coarse_once(const or_params* p, const or_coarse* g, const double* in, double* out) {
    if (g->acnn) {
        if (g->dim == 3) or_acnn3d_forward(g->acnn, p->n, 1, in, out);
        else or_acnn_forward(g->acnn, p->n, 1, in, out);
    } else if (g->cnn) {
        or_cnn_forward(g->cnn, p->n, in, out);
    } else {
        or_fine_any(p, g->dim, g->coarse_steps, in, out);
    }
}

/* The coarse evaluation of a slice: `repeat` applications of the coarse
 * propagator in a row (the composition of the remark after Algorithm 2; 1 is
 * plain G).  tmp holds one field. */
static void or_coarse_eval(const or_params* p, const or_coarse* g, int repeat, const double* in, double* out,
                           double* tmp) {
    size_t m = or_field_len(p, g->dim);
    if (repeat <= 1) { or_coarse_once(p, g, in, out); return; }
    memcpy(tmp, in, sizeof(double) * m);
    for (int r = 0; r < repeat; r++) {
        or_coarse_once(p, g, tmp, out);
        if (r + 1 < repeat) memcpy(tmp, out, sizeof(double) * m);
    }
}

typedef struct { const or_params* p; int dim, c, first; size_t m; const double* in; double* out; } fine_slices_ctx;

/* Fine solves of slices first + [lo, hi) (each one independent). */
static void fine_slices_run(void* vc, long lo, long hi) {
    const fine_slices_ctx* q = (const fine_slices_ctx*)vc;
    for (long t = lo; t < hi; t++) {
        const size_t j = (size_t)(q->first + t);
        or_fine_any(q->p, q->dim, q->c, q->in + j * q->m, q->out + j * q->m);
    }
}

static long or_parareal_g(const or_params* p, const or_coarse* g, int repeat, int s, int c, int kmax, double tol,
                          int literal, const double* u0, double* U, double* res_l2, double* res_max, int* iters);

long or_parareal(const or_params* p, const or_cnn* coarse, int coarse_steps, int s, int c,
                 int kmax, double tol, int literal, const double* u0, double* U,
                 double* res_l2, double* res_max, int* iters) {
    or_coarse g = {coarse, NULL, coarse_steps, 2};
    return or_parareal_g(p, &g, 1, s, c, kmax, tol, literal, u0, U, res_l2, res_max, iters);
}

/* Algorithm 2 with the coarse propagator composed `repeat` times per slice;
 * returns the number of coarse applications (repeat per evaluation). */
long or_parareal_rep(const or_params* p, const or_cnn* coarse, int coarse_steps, int repeat, int s, int c,
                     int kmax, double tol, int literal, const double* u0, double* U,
                     double* res_l2, double* res_max, int* iters) {
    or_coarse g = {coarse, NULL, coarse_steps, 2};
    return or_parareal_g(p, &g, repeat, s, c, kmax, tol, literal, u0, U, res_l2, res_max, iters);
}

/* Algorithm 2 with the ResBlock ACNN (Sec. 3.2) as G. */
long or_parareal_acnn(const or_params* p, const or_acnn* coarse, int repeat, int s, int c, int kmax, double tol,
                      const double* u0, double* U, double* res_l2, double* res_max, int* iters) {
    or_coarse g = {NULL, coarse, 0, 2};
    return or_parareal_g(p, &g, repeat, s, c, kmax, tol, 0, u0, U, res_l2, res_max, iters);
}

/* Algorithm 2 on the periodic cube: the 3D fine step as F, and as G the
 * ResBlock ACNN with 3 x 3 x 3 convolutions (coarse != NULL) or the 3D fine
 * step over coarse_steps steps. */
long or_parareal3d(const or_params* p, const or_acnn* coarse, int coarse_steps, int repeat, int s, int c, int kmax,
                   double tol, const double* u0, double* U, double* res_l2, double* res_max, int* iters) {
    or_coarse g = {NULL, coarse, coarse_steps, 3};
    return or_parareal_g(p, &g, repeat, s, c, kmax, tol, 0, u0, U, res_l2, res_max, iters);
}

static long or_parareal_g(const or_params* p, const or_coarse* gc, int repeat, int s, int c, int kmax, double tol,
                          int literal, const double* u0, double* U, double* res_l2, double* res_max, int* iters) {
    size_t m = or_field_len(p, gc->dim);
    double* Uold = malloc(sizeof(double) * m * (s + 1));
    double* Gold = malloc(sizeof(double) * m * s);
    double* Ff = malloc(sizeof(double) * m * s);
    double* g = malloc(sizeof(double) * m);
    double* gt = malloc(sizeof(double) * m);
    long gcalls = 0;
    if (repeat < 1) repeat = 1;
#define GAPPLY(in, out) do { or_coarse_eval(p, gc, repeat, (in), (out), gt); \
                             gcalls += repeat; } while (0)
    /* k = 0: sequential coarse sweep */
    memcpy(U, u0, sizeof(double) * m);
    for (int j = 0; j < s; j++) {
        GAPPLY(U + j * m, Gold + j * m);
        memcpy(U + (j + 1) * m, Gold + j * m, sizeof(double) * m);
    }
    int k;
    for (k = 1; k <= kmax && k <= s; k++) {
        memcpy(Uold, U, sizeof(double) * m * (s + 1));
        /* fine solves, independent over n = k-1 .. s-1 */
        fine_slices_ctx fq = {p, gc->dim, c, k - 1, m, Uold, Ff};
        or_parallel_for(s - (k - 1), fine_slices_run, &fq);
        /* sequential correction */
        for (int j = k - 1; j < s; j++) {
            if (literal) {
                double* gn = malloc(sizeof(double) * m);
                double* go = malloc(sizeof(double) * m);
                GAPPLY(U + j * m, gn);
                GAPPLY(Uold + j * m, go);
                for (size_t i = 0; i < m; i++) U[(j + 1) * m + i] = Ff[j * m + i] + (gn[i] - go[i]);
                free(gn); free(go);
            } else {
                if (j == k - 1) {
                    /* U^k_{k-1} = U^{k-1}_{k-1}: the new G value is the stored one */
                    for (size_t i = 0; i < m; i++)
                        U[(j + 1) * m + i] = Ff[j * m + i] + (Gold[j * m + i] - Gold[j * m + i]);
                } else {
                    GAPPLY(U + j * m, g);
                    for (size_t i = 0; i < m; i++) U[(j + 1) * m + i] = Ff[j * m + i] + (g[i] - Gold[j * m + i]);
                    memcpy(Gold + j * m, g, sizeof(double) * m);
                }
            }
        }
        or_residual_len(s, m, U, Uold, &res_l2[k], &res_max[k]);
        if (res_l2[k] < tol) break;
    }
    if (k > kmax || k > s) k--;
    *iters = k;
    free(Uold); free(Gold); free(Ff); free(g); free(gt);
#undef GAPPLY
    return gcalls;
}

/* ------------------------------------------------ ResBlock ACNN (Sec. 3.2) */
/* The paper's coarse network: an input convolution 1 -> C, `blocks` residual
 * blocks of two C -> C convolutions, an output convolution C -> 1; tanh after
 * every convolution but the output one; circular padding; then the mACNN mass
 * shift and the bound limiter.  A block maps x to x + tanh(conv2(tanh(conv1(x)))).
 * Parameters: concat of W_in[C][1][3][3], per block W_1, W_2 [C][C][3][3],
 * W_out[1][C][3][3]; biases in the same order (b_in[C], b_1[C], b_2[C],
 * b_out[1]). */
struct or_acnn_s {
    int channels;
    int blocks;
    int mass_fix;   /* 1: add mean(input) - mean(output) */
    int limiter;    /* 1: clamp to [lo, hi] */
    double lo, hi;
    const double* w;
    const double* b;
};

static int acnn_convs(const or_acnn* d) { return 2 + 2 * d->blocks; }

static void acnn_dims(const or_acnn* d, int l, int* cin, int* cout) {
    *cin = (l == 0) ? 1 : d->channels;
    *cout = (l == acnn_convs(d) - 1) ? 1 : d->channels;
}

static void acnn_offsets(const or_acnn* d, int l, int* wo, int* bo) {
    int w = 0, b = 0;
    for (int i = 0; i < l; i++) { int ci, co; acnn_dims(d, i, &ci, &co); w += ci * co * 9; b += co; }
    *wo = w; *bo = b;
}

long or_acnn_param_counts(const or_acnn* d, long* nb) {
    int wo, bo;
    acnn_offsets(d, acnn_convs(d), &wo, &bo);
    if (nb) *nb = bo;
    return wo;
}

/* Saved state of one forward pass: x[0..R] block inputs (x[R] feeds the
 * output conv), h[R] and t[R] the two tanh outputs of each block, o the
 * output conv, s the field after the mass shift (before the limiter). */
typedef struct { double *x, *h, *t, *o, *s; } acnn_saved;

static void acnn_forward_saved(const or_acnn* d, int n, const double* u, double* out, acnn_saved* sv) {
    size_t m = (size_t)n * n;
    int C = d->channels, R = d->blocks;
    int wo, bo;
    acnn_offsets(d, 0, &wo, &bo);
    conv3x3(n, 1, C, d->w + wo, d->b + bo, u, sv->x);
    for (size_t i = 0; i < (size_t)C * m; i++) sv->x[i] = tanh(sv->x[i]);
    for (int r = 0; r < R; r++) {
        double* x = sv->x + (size_t)r * C * m;
        double* xn = sv->x + (size_t)(r + 1) * C * m;
        double* h = sv->h + (size_t)r * C * m;
        double* t = sv->t + (size_t)r * C * m;
        acnn_offsets(d, 1 + 2 * r, &wo, &bo);
        conv3x3(n, C, C, d->w + wo, d->b + bo, x, h);
        for (size_t i = 0; i < (size_t)C * m; i++) h[i] = tanh(h[i]);
        acnn_offsets(d, 2 + 2 * r, &wo, &bo);
        conv3x3(n, C, C, d->w + wo, d->b + bo, h, t);
        for (size_t i = 0; i < (size_t)C * m; i++) { t[i] = tanh(t[i]); xn[i] = x[i] + t[i]; }
    }
    acnn_offsets(d, 1 + 2 * R, &wo, &bo);
    conv3x3(n, C, 1, d->w + wo, d->b + bo, sv->x + (size_t)R * C * m, sv->o);
    double shift = 0.0;
    if (d->mass_fix) {
        double su = 0.0, so = 0.0;
        for (size_t i = 0; i < m; i++) { su += u[i]; so += sv->o[i]; }
        shift = (su - so) / (double)m;
    }
    for (size_t i = 0; i < m; i++) {
        sv->s[i] = sv->o[i] + shift;
        double v = sv->s[i];
        if (d->limiter) v = v < d->lo ? d->lo : (v > d->hi ? d->hi : v);
        out[i] = v;
    }
}

static acnn_saved acnn_alloc(const or_acnn* d, int n) {
    size_t m = (size_t)n * n, C = d->channels, R = d->blocks;
    acnn_saved sv;
    sv.x = malloc(sizeof(double) * (R + 1) * C * m);
    sv.h = malloc(sizeof(double) * (R ? R : 1) * C * m);
    sv.t = malloc(sizeof(double) * (R ? R : 1) * C * m);
    sv.o = malloc(sizeof(double) * m);
    sv.s = malloc(sizeof(double) * m);
    return sv;
}

static void acnn_free(acnn_saved* sv) { free(sv->x); free(sv->h); free(sv->t); free(sv->o); free(sv->s); }

void or_acnn_forward(const or_acnn* d, int n, int batch, const double* u, double* out) {
    size_t m = (size_t)n * n;
    acnn_saved sv = acnn_alloc(d, n);
    for (int p = 0; p < batch; p++) acnn_forward_saved(d, n, u + p * m, out + p * m, &sv);
    acnn_free(&sv);
}

/* dL/dW of one 3x3 circular correlation: gw[o][c][a][e] += sum_ij g[o][i][j] in[c][i+a-1][j+e-1],
 * gb[o] += sum_ij g[o][i][j]. */
static void conv3x3_wgrad(int n, int cin, int cout, const double* in, const double* g, double* gw, double* gb) {
    size_t m = (size_t)n * n;
    for (int o = 0; o < cout; o++) {
        for (size_t i = 0; i < m; i++) gb[o] += g[o * m + i];
        for (int c = 0; c < cin; c++)
            for (int a = 0; a < 3; a++)
                for (int e = 0; e < 3; e++) {
                    double acc = 0.0;
                    for (int i = 0; i < n; i++)
                        for (int j = 0; j < n; j++)
                            acc += g[o * m + (size_t)i * n + j] *
                                   in[c * m + (size_t)((i + a - 1 + n) % n) * n + (j + e - 1 + n) % n];
                    gw[((o * cin + c) * 3 + a) * 3 + e] += acc;
                }
    }
}

/* Adjoint of the correlation with respect to its input: every output
 * gradient scattered back through the stencil (gin is overwritten). */
static void conv3x3_dgrad(int n, int cin, int cout, const double* W, const double* g, double* gin) {
    size_t m = (size_t)n * n;
    memset(gin, 0, sizeof(double) * cin * m);
    for (int o = 0; o < cout; o++)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++) {
                double gv = g[o * m + (size_t)i * n + j];
                for (int c = 0; c < cin; c++)
                    for (int a = 0; a < 3; a++)
                        for (int e = 0; e < 3; e++)
                            gin[c * m + (size_t)((i + a - 1 + n) % n) * n + (j + e - 1 + n) % n] +=
                                W[((o * cin + c) * 3 + a) * 3 + e] * gv;
            }
}

/* Weight and bias gradients of the ACNN, summed over the batch, for
 * gout = dL/d(output) (after the limiter).  gw, gb are overwritten.  The
 * limiter passes the gradient where lo < s < hi (zero where it clamps); the
 * mass shift contributes -mean(g) (its input term does not reach the
 * parameters). */
void or_acnn_backward(const or_acnn* d, int n, int batch, const double* u, const double* gout,
                      double* gw, double* gb) {
    size_t m = (size_t)n * n;
    int C = d->channels, R = d->blocks;
    long nb, nw = or_acnn_param_counts(d, &nb);
    memset(gw, 0, sizeof(double) * nw);
    memset(gb, 0, sizeof(double) * nb);
    acnn_saved sv = acnn_alloc(d, n);
    double* out = malloc(sizeof(double) * m);
    double* go = malloc(sizeof(double) * m);
    double* gx = malloc(sizeof(double) * C * m);
    double* gz = malloc(sizeof(double) * C * m);
    double* gh = malloc(sizeof(double) * C * m);
    for (int p = 0; p < batch; p++) {
        acnn_forward_saved(d, n, u + p * m, out, &sv);
        for (size_t i = 0; i < m; i++) {
            double g = gout[p * m + i];
            if (d->limiter && !(sv.s[i] > d->lo && sv.s[i] < d->hi)) g = 0.0;
            go[i] = g;
        }
        if (d->mass_fix) {
            double mean = 0.0;
            for (size_t i = 0; i < m; i++) mean += go[i];
            mean /= (double)m;
            for (size_t i = 0; i < m; i++) go[i] -= mean;
        }
        int wo, bo;
        acnn_offsets(d, 1 + 2 * R, &wo, &bo);
        conv3x3_wgrad(n, C, 1, sv.x + (size_t)R * C * m, go, gw + wo, gb + bo);
        conv3x3_dgrad(n, C, 1, d->w + wo, go, gx);
        for (int r = R - 1; r >= 0; r--) {
            const double* x = sv.x + (size_t)r * C * m;
            const double* h = sv.h + (size_t)r * C * m;
            const double* t = sv.t + (size_t)r * C * m;
            for (size_t i = 0; i < (size_t)C * m; i++) gz[i] = gx[i] * (1.0 - t[i] * t[i]);
            acnn_offsets(d, 2 + 2 * r, &wo, &bo);
            conv3x3_wgrad(n, C, C, h, gz, gw + wo, gb + bo);
            conv3x3_dgrad(n, C, C, d->w + wo, gz, gh);
            for (size_t i = 0; i < (size_t)C * m; i++) gz[i] = gh[i] * (1.0 - h[i] * h[i]);
            acnn_offsets(d, 1 + 2 * r, &wo, &bo);
            conv3x3_wgrad(n, C, C, x, gz, gw + wo, gb + bo);
            conv3x3_dgrad(n, C, C, d->w + wo, gz, gh);
            for (size_t i = 0; i < (size_t)C * m; i++) gx[i] += gh[i];
        }
        for (size_t i = 0; i < (size_t)C * m; i++) gz[i] = gx[i] * (1.0 - sv.x[i] * sv.x[i]);
        acnn_offsets(d, 0, &wo, &bo);
        conv3x3_wgrad(n, 1, C, u + p * m, gz, gw + wo, gb + bo);
    }
    acnn_free(&sv);
    free(out); free(go); free(gx); free(gz); free(gh);
}

/* Scheme-residual loss (Eq. loss_ACN) of a batch of pairs (U_n, U_{n+1}) with
 * the time step p->dt:  r = U1 - U0 - dt/2 (eps^2 Lap_h (U1 + U0) + f(U1) + f(U0)
 * - g(U1) - g(U0)),  g(U) = mean f(U) for the mass-conserving variant, 0 for
 * the classic one;  L = sum r^2 / (batch N^2).  If grad != NULL it receives
 * dL/dU1 = 2/(batch N^2) (r - dt/2 (eps^2 Lap_h r + f'(U1) r - [mass] f'(U1) mean r))
 * (Lap_h is symmetric; d g(U1)/dU1 = f'(U1)/N^2 at every entry). */
double or_loss_acn(const or_params* p, int batch, const double* U0, const double* U1, double* grad) {
    int n = p->n;
    size_t m = (size_t)n * n;
    double h = p->length / n, e2 = p->eps * p->eps, dt = p->dt;
    double* s = malloc(sizeof(double) * m);
    double* ls = malloc(sizeof(double) * m);
    double* r = malloc(sizeof(double) * m);
    double total = 0.0;
    for (int b = 0; b < batch; b++) {
        const double* a = U0 + b * m;
        const double* c = U1 + b * m;
        double g0 = 0.0, g1 = 0.0;
        if (p->variant == 1) {
            for (size_t i = 0; i < m; i++) { g0 += f_dw(a[i]); g1 += f_dw(c[i]); }
            g0 /= (double)m; g1 /= (double)m;
        }
        for (size_t i = 0; i < m; i++) s[i] = a[i] + c[i];
        apply_lap(n, h, s, ls);
        double rmean = 0.0;
        for (size_t i = 0; i < m; i++) {
            r[i] = c[i] - a[i] - 0.5 * dt * (e2 * ls[i] + f_dw(c[i]) + f_dw(a[i]) - g1 - g0);
            total += r[i] * r[i];
            rmean += r[i];
        }
        rmean /= (double)m;
        if (grad) {
            double scale = 2.0 / ((double)batch * (double)m);
            apply_lap(n, h, r, ls);
            for (size_t i = 0; i < m; i++) {
                double fp = fprime_dw(c[i]);
                double jr = e2 * ls[i] + fp * r[i] - (p->variant == 1 ? fp * rmean : 0.0);
                grad[b * m + i] = scale * (r[i] - 0.5 * dt * jr);
            }
        }
    }
    free(s); free(ls); free(r);
    return total / ((double)batch * (double)m);
}

/* One Adam update (Kingma & Ba, Algorithm 1) of `count` parameters at step t >= 1:
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, w -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps). */
void or_adam(double* w, const double* g, double* mo, double* vo, long count, double lr, double b1, double b2,
             double eps, int t) {
    double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long i = 0; i < count; i++) {
        mo[i] = b1 * mo[i] + (1.0 - b1) * g[i];
        vo[i] = b2 * vo[i] + (1.0 - b2) * g[i] * g[i];
        w[i] -= lr * (mo[i] / c1) / (sqrt(vo[i] / c2) + eps);
    }
}

/* Algorithm 1: training of the ACNN with the scheme-residual loss.
 * For each epoch e the R initial conditions are visited in the order
 * perm[e][0..R-1], cut into R/q subsets of q.  For each subset, U starts at
 * its q initial conditions; for each of `steps` time steps, b inner updates
 * each predict U1 = G(U; theta), take the loss of (U, U1) and one Adam step
 * on theta; U then becomes the U1 of the last inner update.  w, b (the
 * network's parameters, updated in place), m, v (Adam moments, w then b) and
 * *t (Adam step count) carry over between calls.  losses receives one value
 * per update, in order (epochs * (R/q) * steps * b_inner). */
void or_acnn_train(const or_params* p, or_acnn* d, double* w, double* bias, int R, const double* U0s,
                   const int* perm, int q, int steps, int b_inner, int epochs, double lr, double b1, double b2,
                   double aeps, double* mo, double* vo, int* t, double* losses) {
    int n = p->n;
    size_t m = (size_t)n * n;
    long nb, nw = or_acnn_param_counts(d, &nb);
    d->w = w;
    d->b = bias;
    double* U = malloc(sizeof(double) * q * m);
    double* U1 = malloc(sizeof(double) * q * m);
    double* g = malloc(sizeof(double) * q * m);
    double* gw = malloc(sizeof(double) * (nw + nb));
    long li = 0;
    for (int e = 0; e < epochs; e++)
        for (int sub = 0; sub < R / q; sub++) {
            for (int j = 0; j < q; j++) memcpy(U + j * m, U0s + (size_t)perm[e * R + sub * q + j] * m, sizeof(double) * m);
            for (int st = 0; st < steps; st++) {
                for (int k = 0; k < b_inner; k++) {
                    or_acnn_forward(d, n, q, U, U1);
                    losses[li++] = or_loss_acn(p, q, U, U1, g);
                    or_acnn_backward(d, n, q, U, g, gw, gw + nw);
                    *t += 1;
                    or_adam(w, gw, mo, vo, nw, lr, b1, b2, aeps, *t);
                    or_adam(bias, gw + nw, mo + nw, vo + nw, nb, lr, b1, b2, aeps, *t);
                }
                memcpy(U, U1, sizeof(double) * q * m);
            }
        }
    free(U); free(U1); free(g); free(gw);
}

/* ---------------------------------------------------------------- 3D ---- */
/* The model on the periodic cube (d = 3, Sec. 2; the 3D experiments of
 * Sec. 4): fields u[i][j][k] row-major with k fastest, N^3 points, h = L/N,
 * Lap_h the periodic 7-point stencil with symbol
 * -(4/h^2)(sin^2(pi a/N) + sin^2(pi b/N) + sin^2(pi c/N)). */

/* 3D transform: along k (contiguous), then j, then i. */
void or_fft3d(cplx* x, int n, int sign) {
    size_t nn = (size_t)n * n;
    cplx* line = malloc(sizeof(cplx) * n);
    for (size_t r = 0; r < nn; r++) or_fft1d(x + r * n, n, sign);
    for (int i = 0; i < n; i++)
        for (int k = 0; k < n; k++) {
            for (int j = 0; j < n; j++) line[j] = x[i * nn + (size_t)j * n + k];
            or_fft1d(line, n, sign);
            for (int j = 0; j < n; j++) x[i * nn + (size_t)j * n + k] = line[j];
        }
    for (size_t jk = 0; jk < nn; jk++) {
        for (int i = 0; i < n; i++) line[i] = x[i * nn + jk];
        or_fft1d(line, n, sign);
        for (int i = 0; i < n; i++) x[i * nn + jk] = line[i];
    }
    free(line);
}

void or_fft3d_ri(double* xri, int n, int sign) { or_fft3d((cplx*)xri, n, sign); }

static double lap_symbol3(int a, int b, int c, int n, double h) {
    double sa = sin(PI * a / n), sb = sin(PI * b / n), sc = sin(PI * c / n);
    return -(4.0 / (h * h)) * (sa * sa + sb * sb + sc * sc);
}

/* Solve ((1 + S dt) I - dt eps^2 Lap_h) v = r on the cube by the 3D DFT. */
void or_solve_A3(const or_params* p, const double* r, double* v) {
    int n = p->n;
    size_t m = (size_t)n * n * n;
    double h = p->length / n;
    cplx* z = malloc(sizeof(cplx) * m);
    for (size_t i = 0; i < m; i++) z[i] = r[i];
    or_fft3d(z, n, -1);
    for (int a = 0; a < n; a++)
        for (int b = 0; b < n; b++)
            for (int c = 0; c < n; c++) {
                double D = 1.0 + p->S * p->dt - p->dt * p->eps * p->eps * lap_symbol3(a, b, c, n, h);
                z[((size_t)a * n + b) * n + c] /= D;
            }
    or_fft3d(z, n, +1);
    for (size_t i = 0; i < m; i++) v[i] = creal(z[i]) / (double)m;
    free(z);
}

/* The stabilised semi-implicit step of or_fine_step on the cube. */
void or_fine3d_step(const or_params* p, const double* u, double* out) {
    size_t m = (size_t)p->n * p->n * p->n;
    double beta = 0.0;
    if (p->variant == 1) {
        for (size_t i = 0; i < m; i++) beta += f_dw(u[i]);
        beta /= (double)m;
    }
    double* r = malloc(sizeof(double) * m);
    for (size_t i = 0; i < m; i++) r[i] = (1.0 + p->S * p->dt) * u[i] + p->dt * (f_dw(u[i]) - beta);
    or_solve_A3(p, r, out);
    free(r);
}

void or_fine3d_propagate(const or_params* p, int steps, const double* u, double* out) {
    size_t m = (size_t)p->n * p->n * p->n;
    double* a = malloc(sizeof(double) * m);
    memcpy(a, u, sizeof(double) * m);
    for (int s = 0; s < steps; s++) {
        or_fine3d_step(p, a, out);
        memcpy(a, out, sizeof(double) * m);
    }
    if (steps == 0) memcpy(out, u, sizeof(double) * m);
    free(a);
}

/* 7-point periodic Laplacian applied directly. */
void or_lap3(int n, double h, const double* u, double* out) {
    size_t nn = (size_t)n * n;
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            for (int k = 0; k < n; k++) {
                size_t c = i * nn + (size_t)j * n + k;
                double s = u[((i + 1) % n) * nn + (size_t)j * n + k] + u[((i + n - 1) % n) * nn + (size_t)j * n + k] +
                           u[i * nn + (size_t)((j + 1) % n) * n + k] + u[i * nn + (size_t)((j + n - 1) % n) * n + k] +
                           u[i * nn + (size_t)j * n + (k + 1) % n] + u[i * nn + (size_t)j * n + (k + n - 1) % n];
                out[c] = (s - 6.0 * u[c]) / (h * h);
            }
}

/* ------------------------------------------- ResBlock ACNN on the cube ---- */
/* The network of or_acnn_forward with 3 x 3 x 3 circular convolutions (the
 * 3D experiments of Sec. 4): parameters W_l[cout][cin][3][3][3] concatenated
 * in the same layer order, biases as in 2D.  Fields [n][n][n], last index
 * fastest. */
static void acnn3_offsets(const or_acnn* d, int l, int* wo, int* bo) {
    int w = 0, b = 0;
    for (int i = 0; i < l; i++) { int ci, co; acnn_dims(d, i, &ci, &co); w += ci * co * 27; b += co; }
    *wo = w; *bo = b;
}

long or_acnn3d_param_counts(const or_acnn* d, long* nb) {
    int wo, bo;
    acnn3_offsets(d, acnn_convs(d), &wo, &bo);
    if (nb) *nb = bo;
    return wo;
}

/* out[o][i][j][k] = b[o] + sum_{c,a,e,g} W[o][c][a][e][g] in[c][i+a-1][j+e-1][k+g-1] (indices mod n). */
static void conv3x3x3(int n, int cin, int cout, const double* W, const double* b, const double* in, double* out) {
    size_t m = (size_t)n * n * n, nn = (size_t)n * n;
    for (int o = 0; o < cout; o++)
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                for (int k = 0; k < n; k++) {
                    double acc = b[o];
                    for (int c = 0; c < cin; c++)
                        for (int a = 0; a < 3; a++)
                            for (int e = 0; e < 3; e++)
                                for (int g = 0; g < 3; g++) {
                                    size_t ii = (i + a - 1 + n) % n, jj = (j + e - 1 + n) % n, kk = (k + g - 1 + n) % n;
                                    acc += W[(((o * cin + c) * 3 + a) * 3 + e) * 3 + g] * in[c * m + ii * nn + jj * n + kk];
                                }
                    out[o * m + (size_t)i * nn + (size_t)j * n + k] = acc;
                }
}

static void acnn3d_one(const or_acnn* d, int n, const double* u, double* out, double* x, double* h, double* t,
                       double* o) {
    size_t m = (size_t)n * n * n;
    int C = d->channels, R = d->blocks;
    int wo, bo;
    acnn3_offsets(d, 0, &wo, &bo);
    conv3x3x3(n, 1, C, d->w + wo, d->b + bo, u, x);
    for (size_t i = 0; i < (size_t)C * m; i++) x[i] = tanh(x[i]);
    for (int r = 0; r < R; r++) {
        acnn3_offsets(d, 1 + 2 * r, &wo, &bo);
        conv3x3x3(n, C, C, d->w + wo, d->b + bo, x, h);
        for (size_t i = 0; i < (size_t)C * m; i++) h[i] = tanh(h[i]);
        acnn3_offsets(d, 2 + 2 * r, &wo, &bo);
        conv3x3x3(n, C, C, d->w + wo, d->b + bo, h, t);
        for (size_t i = 0; i < (size_t)C * m; i++) x[i] += tanh(t[i]);
    }
    acnn3_offsets(d, 1 + 2 * R, &wo, &bo);
    conv3x3x3(n, C, 1, d->w + wo, d->b + bo, x, o);
    double shift = 0.0;
    if (d->mass_fix) {
        double su = 0.0, so = 0.0;
        for (size_t i = 0; i < m; i++) { su += u[i]; so += o[i]; }
        shift = (su - so) / (double)m;
    }
    for (size_t i = 0; i < m; i++) {
        double v = o[i] + shift;
        if (d->limiter) v = v < d->lo ? d->lo : (v > d->hi ? d->hi : v);
        out[i] = v;
    }
}

void or_acnn3d_forward(const or_acnn* d, int n, int batch, const double* u, double* out) {
    size_t m = (size_t)n * n * n;
    int C = d->channels;
    double* x = malloc(sizeof(double) * C * m);
    double* h = malloc(sizeof(double) * C * m);
    double* t = malloc(sizeof(double) * C * m);
    double* o = malloc(sizeof(double) * m);
    for (int p = 0; p < batch; p++) acnn3d_one(d, n, u + p * m, out + p * m, x, h, t, o);
    free(x); free(h); free(t); free(o);
}
