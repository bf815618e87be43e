/*
 * Lid-driven cavity, vorticity / stream-function form: plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, deliberately plain reference
 * that the CUDA library is checked against.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it; the library never does,
 * and it shares no source with the library.
 *
 * Method: N. Cardoso and P. Bicudo, "Time dependent simulation of the Driven
 * Lid Cavity at High Reynolds Number" (arXiv:0809.3098).  Equation numbers
 * below follow the paper's numbering:
 *   Eq. (1)-(5)   vorticity, stream function, vorticity transport (Sec. 2)
 *   Eq. (7)-(8)   explicit update and the spatial operator L(omega) (Sec. 3)
 *   Eq. (9)-(13)  SSPRK(5,4) of Ruuth and Spiteri in Shu-Osher form (Sec. 3)
 *   Eq. (14)      fourth-order compact Poisson equation (Sec. 3)
 *   Eq. (15)-(21) SOR update with the terms A, B, C and a, b, c (Sec. 3)
 *   Eq. (22)      velocities from psi (Sec. 3)
 *   Eq. (23)-(25) wall conditions and Thom's wall vorticity (Sec. 3.1)
 *   Eq. (26)-(27) RES_psi, RES_omega steady-state monitors (Sec. 3.2)
 *
 * Grid: N intervals per side, (N+1) x (N+1) nodes, h = 1/N, array index
 * j*(N+1) + i with i the x index (0 = left wall, N = right wall) and j the y
 * index (0 = bottom wall, N = lid).  The paper counts nodes 1..n; here wall
 * nodes are i or j equal to 0 or N.
 *
 * Readings taken where the paper is silent (each one is listed with its
 * reason in the project's design notes):
 *   R1  N counts intervals, h = 1/N.
 *   R2  Thom's formula uses h^2 on every wall (Eq. 25 mixes dx and dy; here
 *       dx = dy = h, so nothing depends on it).
 *   R3  the four corner nodes hold psi = 0 and omega = 0; no stencil reads them
 *       except the compact operator's diagonal psi terms, where psi = 0.
 *   R4  Eq. (10) prints the omega^(1) weight as 0.555626506348765; the weights
 *       of every stage sum to one, so this is read as 0.555629506348765.
 *       Eq. (9)'s 0.39175222657 is carried to 0.391752226571890.
 *   R5  wall vorticity is not integrated by the Runge-Kutta stages: Thom's
 *       formula sets it after every Poisson solve and it is held while L is
 *       evaluated.
 *   R6  the compact right-hand side B (Eq. 17) at wall-adjacent nodes uses the
 *       wall vorticity of the previous solve (lagged); the coupling is not
 *       iterated.
 *   R7  the Poisson equation is solved to a relative residual
 *       ||f - L_h psi||_2 <= tol ||f||_2 over interior nodes, checked after
 *       every multigrid V-cycle, at least one cycle per solve, warm-started
 *       from the previous solve; the SOR iteration of Eq. (15) is used as the
 *       smoother with colour ordering (red-black for the 5-point operator, four
 *       colours (i mod 2, j mod 2) for the compact operator).
 *   R8  psi(omega^{n+1}) is solved at the end of each step, so a step makes
 *       five solves and the next step's first stage reuses it.
 *   R12 multigrid halves a level while its interval count is even and >= 4;
 *       the coarsest level (2, 3, 5 or 7 intervals) gets nuc smoothing sweeps.
 *   R15 with the option coarse_direct (default on) the V-cycle instead ends
 *       at the first level below the finest with at most 16 intervals, where
 *       the level's equation is solved exactly (a direct solve of the dense
 *       system; at most 225 unknowns).
 *   R13 the alternative solver "SOR" is Eq. (15) on its own, swept in the
 *       order its n / n+1 superscripts fix (i outer, j inner), with the
 *       stopping test of R7 after every sor_sweeps sweeps.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_OP_5PT 0
#define OR_OP_COMPACT 1
#define OR_SOLVER_MG 0
#define OR_SOLVER_SOR 1

#define OR_OK 0
#define OR_ERR_ARG -1
#define OR_ERR_NOCONV -3
#define OR_ERR_NONFINITE -4

#define AT(N, i, j) ((size_t)(j) * (size_t)((N) + 1) + (size_t)(i))

/* Threads for the loops whose iterations are independent: a colour phase of
 * the smoother (no node of a colour reads another of that colour), the
 * operator, residual, restriction, prolongation, right-hand side, L(omega)
 * and the Runge-Kutta combination (each output node written by one
 * iteration from inputs no iteration writes).  Every node is computed by the
 * same expression whatever the thread count, and the reductions (norms,
 * monitors) and the lexicographic SOR sweep stay serial, so the results are
 * bit-identical for any count.  Default 1; set by or_set_threads.  Built
 * without OpenMP the pragmas are ignored and the count has no effect. */
static int or_threads = 1;

void or_set_threads(int n) { or_threads = n < 1 ? 1 : n; }
int or_get_threads(void) { return or_threads; }

/* Whether a loop of n rows is worth splitting over threads. */
static int or_par(int n) { return or_threads > 1 && n >= 64; }

/* ------------------------------------------------------------------------ */
/* SSPRK(5,4) coefficients, Eqs. (9)-(13), in Shu-Osher form:
 *   y_s = sum_{k<s} ( alpha[s][k] y_k + dt beta[s][k] L(y_k) ),  s = 1..5,
 * with y_0 = omega^n and y_5 = omega^{n+1}.  Reading R4 applies to
 * alpha[2][1] and beta[1][0]. */
static const double SSP_ALPHA[6][5] = {
    {0, 0, 0, 0, 0},
    {1.0, 0, 0, 0, 0},
    {0.444370493651235, 0.555629506348765, 0, 0, 0},
    {0.620101851488403, 0, 0.379898148511597, 0, 0},
    {0.178079954393132, 0, 0, 0.821920045606868, 0},
    {0, 0, 0.517231671970585, 0.096059710526147, 0.386708617503269},
};
static const double SSP_BETA[6][5] = {
    {0, 0, 0, 0, 0},
    {0.391752226571890, 0, 0, 0, 0},
    {0, 0.368410593050371, 0, 0, 0},
    {0, 0, 0.251891774271694, 0, 0},
    {0, 0, 0, 0.544974750228521, 0},
    {0, 0, 0, 0.063692468666290, 0.226007483236906},
};

/* Copies the coefficient tables out (row s = 0..5, column k = 0..4). */
void or_ssprk54_coefficients(double *alpha_out, double *beta_out) {
    for (int s = 0; s < 6; ++s)
        for (int k = 0; k < 5; ++k) {
            alpha_out[s * 5 + k] = SSP_ALPHA[s][k];
            beta_out[s * 5 + k] = SSP_BETA[s][k];
        }
}

/* One SSPRK(5,4) step of y' = L(y) for a vector of n unknowns, Eqs. (9)-(13).
 * L(user, s, y_s, out) evaluates L at stage input s (0..4).  work holds
 * 11*n doubles (six stage values and five L values).  On return y = y_5. */
typedef void (*or_L_fn)(void *user, int stage, const double *y, double *out);

void or_ssprk54_step(int n, double *y, double dt, or_L_fn L, void *user, double *work) {
    double *Y[6], *LY[5];
    for (int s = 0; s < 6; ++s) Y[s] = work + (size_t)s * n;
    for (int s = 0; s < 5; ++s) LY[s] = work + (size_t)(6 + s) * n;
    memcpy(Y[0], y, sizeof(double) * n);
    for (int s = 1; s <= 5; ++s) {
        L(user, s - 1, Y[s - 1], LY[s - 1]);
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(n / 1024))
        for (int m = 0; m < n; ++m) {
            double acc = 0.0;
            for (int k = 0; k < s; ++k) {
                if (SSP_ALPHA[s][k] != 0.0) acc += SSP_ALPHA[s][k] * Y[k][m];
                if (SSP_BETA[s][k] != 0.0) acc += SSP_BETA[s][k] * dt * LY[k][m];
            }
            Y[s][m] = acc;
        }
    }
    memcpy(y, Y[5], sizeof(double) * n);
}

/* ------------------------------------------------------------------------ */
/* Poisson problem.  Terms of Eqs. (16)-(21) with dx = dy = h:
 *   b = 1/dx^2, c = 1/dy^2, a = b + c,
 *   A = b (psi_E + psi_W) + c (psi_N + psi_S),
 *   B = (omega_E + omega_N + 8 omega_P + omega_W + omega_S) / 12,
 *   C = (a/12) (psi_NE - 2 psi_N + psi_NW - 2 psi_E - 2 psi_W + psi_SE
 *               - 2 psi_S + psi_SW).
 * At beta = 1 the fixed point of Eq. (15) is (5/3) a psi = A + B + C, i.e.
 *   L_h psi := A + C - (5/3) a psi = f,   f = -B,
 * the compact fourth-order discretisation of Eq. (14).  The plain 5-point
 * operator of Eq. (3) is L_h psi := A - 2 a psi = f with f = -omega_P.
 * A coarse multigrid level solves the same operator with its own h and a
 * general right-hand side f (the restricted residual), i.e. B = -f. */

/* f at interior nodes from omega (walls of f are zero). */
void or_poisson_rhs(int N, int op, const double *omega, double *f) {
    memset(f, 0, sizeof(double) * (size_t)(N + 1) * (N + 1));
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
            if (op == OR_OP_COMPACT) {
                double B = (omega[AT(N, i + 1, j)] + omega[AT(N, i, j + 1)] + 8.0 * omega[AT(N, i, j)] +
                            omega[AT(N, i - 1, j)] + omega[AT(N, i, j - 1)]) / 12.0;
                f[AT(N, i, j)] = -B;
            } else {
                f[AT(N, i, j)] = -omega[AT(N, i, j)];
            }
        }
}

static double term_A(int N, double b, double c, const double *p, int i, int j) {
    return b * (p[AT(N, i + 1, j)] + p[AT(N, i - 1, j)]) + c * (p[AT(N, i, j + 1)] + p[AT(N, i, j - 1)]);
}

static double term_C(int N, double a, const double *p, int i, int j) {
    return a / 12.0 *
           (p[AT(N, i + 1, j + 1)] - 2.0 * p[AT(N, i, j + 1)] + p[AT(N, i - 1, j + 1)] - 2.0 * p[AT(N, i + 1, j)] -
            2.0 * p[AT(N, i - 1, j)] + p[AT(N, i + 1, j - 1)] - 2.0 * p[AT(N, i, j - 1)] + p[AT(N, i - 1, j - 1)]);
}

/* out = L_h psi at interior nodes (walls of out are zero). */
void or_apply_operator(int N, int op, const double *psi, double *out) {
    double h = 1.0 / N, b = 1.0 / (h * h), c = 1.0 / (h * h), a = b + c;
    memset(out, 0, sizeof(double) * (size_t)(N + 1) * (N + 1));
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
            double A = term_A(N, b, c, psi, i, j);
            if (op == OR_OP_COMPACT)
                out[AT(N, i, j)] = A + term_C(N, a, psi, i, j) - 5.0 / 3.0 * a * psi[AT(N, i, j)];
            else
                out[AT(N, i, j)] = A - 2.0 * a * psi[AT(N, i, j)];
        }
}

/* r = f - L_h psi at interior nodes. */
void or_residual(int N, int op, const double *psi, const double *f, double *r) {
    or_apply_operator(N, op, psi, r);
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) r[AT(N, i, j)] = f[AT(N, i, j)] - r[AT(N, i, j)];
}

/* Does node (i, j) belong to colour `colour`?  5-point: red = (i+j) even is
 * colour 0, black colour 1.  Compact: colour = (i mod 2) + 2 (j mod 2), so no
 * node shares a colour with any of its eight neighbours. */
static int in_colour(int op, int colour, int i, int j) {
    if (op == OR_OP_COMPACT) return (i % 2) + 2 * (j % 2) == colour;
    return (i + j) % 2 == colour;
}

/* nsweeps colour-ordered sweeps of the SOR update, Eq. (15):
 *   compact: psi <- (3/5)(beta/a)(A + B + C) + (1 - beta) psi,  B = -f
 *   5-point: psi <- (1/2)(beta/a)(A + B) + (1 - beta) psi,       B = -f
 * Within a colour no node reads another node of the same colour, so updating
 * a colour in place is the same as updating it all at once. */
void or_smooth(int N, int op, double *psi, const double *f, double beta, int nsweeps) {
    double h = 1.0 / N, b = 1.0 / (h * h), c = 1.0 / (h * h), a = b + c;
    int ncolours = op == OR_OP_COMPACT ? 4 : 2;
    for (int s = 0; s < nsweeps; ++s)
        for (int colour = 0; colour < ncolours; ++colour)
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
            for (int j = 1; j < N; ++j)
                for (int i = 1; i < N; ++i) {
                    if (!in_colour(op, colour, i, j)) continue;
                    double A = term_A(N, b, c, psi, i, j);
                    double B = -f[AT(N, i, j)];
                    double old = psi[AT(N, i, j)];
                    if (op == OR_OP_COMPACT)
                        psi[AT(N, i, j)] = 3.0 / 5.0 * beta / a * (A + B + term_C(N, a, psi, i, j)) + (1.0 - beta) * old;
                    else
                        psi[AT(N, i, j)] = 0.5 * beta / a * (A + B) + (1.0 - beta) * old;
                }
}

/* nsweeps sweeps of the SOR update, Eq. (15), in the order its superscripts
 * fix.  At node (i, j) the equation takes psi at (i-1, j-1), (i-1, j),
 * (i-1, j+1) and (i, j-1) from the current sweep (n+1) and psi at (i+1, j-1),
 * (i+1, j), (i+1, j+1) and (i, j+1) from the previous one (n): i is the outer
 * (slow) loop and j the inner (fast) loop, and updating in place in that
 * order is exactly the method.  Same node formula as or_smooth. */
void or_sor_lex(int N, int op, double *psi, const double *f, double beta, int nsweeps) {
    double h = 1.0 / N, b = 1.0 / (h * h), c = 1.0 / (h * h), a = b + c;
    for (int s = 0; s < nsweeps; ++s)
        for (int i = 1; i < N; ++i)
            for (int j = 1; j < N; ++j) {
                double A = term_A(N, b, c, psi, i, j);
                double B = -f[AT(N, i, j)];
                double old = psi[AT(N, i, j)];
                if (op == OR_OP_COMPACT)
                    psi[AT(N, i, j)] = 3.0 / 5.0 * beta / a * (A + B + term_C(N, a, psi, i, j)) + (1.0 - beta) * old;
                else
                    psi[AT(N, i, j)] = 0.5 * beta / a * (A + B) + (1.0 - beta) * old;
            }
}

/* Full-weighting restriction of a fine interior field (Nf intervals) onto the
 * coarse grid (Nf/2 intervals): weights 1/16 [1 2 1; 2 4 2; 1 2 1]. */
void or_restrict(int Nf, const double *rf, double *fc) {
    int Nc = Nf / 2;
    memset(fc, 0, sizeof(double) * (size_t)(Nc + 1) * (Nc + 1));
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(Nc))
    for (int J = 1; J < Nc; ++J)
        for (int I = 1; I < Nc; ++I) {
            int i = 2 * I, j = 2 * J;
            double centre = rf[AT(Nf, i, j)];
            double edges = rf[AT(Nf, i + 1, j)] + rf[AT(Nf, i - 1, j)] + rf[AT(Nf, i, j + 1)] + rf[AT(Nf, i, j - 1)];
            double corners = rf[AT(Nf, i + 1, j + 1)] + rf[AT(Nf, i - 1, j + 1)] + rf[AT(Nf, i + 1, j - 1)] +
                             rf[AT(Nf, i - 1, j - 1)];
            fc[AT(Nc, I, J)] = (4.0 * centre + 2.0 * edges + corners) / 16.0;
        }
}

/* Bilinear prolongation of a coarse correction ec (zero on the walls), added
 * to the fine field psi at interior nodes. */
void or_prolong_add(int Nc, const double *ec, double *psi) {
    int Nf = 2 * Nc;
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(Nf))
    for (int j = 1; j < Nf; ++j)
        for (int i = 1; i < Nf; ++i) {
            int I = i / 2, J = j / 2;
            double e;
            if (i % 2 == 0 && j % 2 == 0)
                e = ec[AT(Nc, I, J)];
            else if (i % 2 == 1 && j % 2 == 0)
                e = 0.5 * (ec[AT(Nc, I, J)] + ec[AT(Nc, I + 1, J)]);
            else if (i % 2 == 0 && j % 2 == 1)
                e = 0.5 * (ec[AT(Nc, I, J)] + ec[AT(Nc, I, J + 1)]);
            else
                e = 0.25 * (ec[AT(Nc, I, J)] + ec[AT(Nc, I + 1, J)] + ec[AT(Nc, I, J + 1)] + ec[AT(Nc, I + 1, J + 1)]);
            psi[AT(Nf, i, j)] += e;
        }
}

/* 2-norm over interior nodes. */
static double interior_norm2(int N, const double *x) {
    double s = 0.0;
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) s += x[AT(N, i, j)] * x[AT(N, i, j)];
    return sqrt(s);
}

static size_t nodes_of(int n) { return (size_t)(n + 1) * (n + 1); }

/* ------------------------------------------------------------------------ */
/* Exact solve of L_h psi = f on one grid of n intervals (reading R15).  The
 * matrix M = -L_h of the (n-1)^2 interior unknowns (numbered i - 1 + (j - 1)
 * (n - 1)) is built column by column by applying or_apply_operator to unit
 * vectors; it is symmetric positive definite, so it is factorised once as
 * M = G G^T (Cholesky, G lower triangular, row-major in chol[]), and each
 * solve is the forward substitution G y = -f followed by the back
 * substitution G^T psi = y. */
typedef struct {
    int n, op, m2;
    double *chol;
} or_direct;

static int direct_init(or_direct *d, int n, int op) {
    int m = n - 1, m2 = m * m;
    d->n = n;
    d->op = op;
    d->m2 = m2;
    d->chol = calloc((size_t)m2 * m2, sizeof(double));
    double *e = calloc(nodes_of(n), sizeof(double)), *Le = calloc(nodes_of(n), sizeof(double));
    double *M = d->chol;
    for (int k = 0; k < m2; ++k) {
        e[AT(n, 1 + k % m, 1 + k / m)] = 1.0;
        or_apply_operator(n, op, e, Le);
        e[AT(n, 1 + k % m, 1 + k / m)] = 0.0;
        for (int r = 0; r < m2; ++r) M[(size_t)r * m2 + k] = -Le[AT(n, 1 + r % m, 1 + r / m)];
    }
    free(e);
    free(Le);
    /* Cholesky in place: column by column, G[k][k] = sqrt(M[k][k] - sum G[k][q]^2),
     * G[r][k] = (M[r][k] - sum G[r][q] G[k][q]) / G[k][k] for r > k. */
    for (int k = 0; k < m2; ++k) {
        double dk = M[(size_t)k * m2 + k];
        for (int q = 0; q < k; ++q) dk -= M[(size_t)k * m2 + q] * M[(size_t)k * m2 + q];
        if (!(dk > 0.0)) return OR_ERR_ARG;
        dk = sqrt(dk);
        M[(size_t)k * m2 + k] = dk;
        for (int r = k + 1; r < m2; ++r) {
            double v = M[(size_t)r * m2 + k];
            for (int q = 0; q < k; ++q) v -= M[(size_t)r * m2 + q] * M[(size_t)k * m2 + q];
            M[(size_t)r * m2 + k] = v / dk;
        }
        for (int c = k + 1; c < m2; ++c) M[(size_t)k * m2 + c] = 0.0;
    }
    return OR_OK;
}

static void direct_free(or_direct *d) {
    free(d->chol);
    d->chol = NULL;
}

/* psi = L_h^{-1} f at interior nodes (walls of psi untouched). */
static void direct_solve(const or_direct *d, const double *f, double *psi) {
    int n = d->n, m = n - 1, m2 = d->m2;
    const double *G = d->chol;
    double *y = malloc(sizeof(double) * m2);
    for (int r = 0; r < m2; ++r) {
        double v = -f[AT(n, 1 + r % m, 1 + r / m)];
        for (int q = 0; q < r; ++q) v -= G[(size_t)r * m2 + q] * y[q];
        y[r] = v / G[(size_t)r * m2 + r];
    }
    for (int r = m2 - 1; r >= 0; --r) {
        double v = y[r];
        for (int q = r + 1; q < m2; ++q) v -= G[(size_t)q * m2 + r] * y[q];
        y[r] = v / G[(size_t)r * m2 + r];
    }
    for (int r = 0; r < m2; ++r) psi[AT(n, 1 + r % m, 1 + r / m)] = y[r];
    free(y);
}

/* Stand-alone exact solve for the pins. */
int or_direct_solve(int n, int op, const double *f, double *psi) {
    if (n < 2 || n > 64) return OR_ERR_ARG;
    or_direct d;
    int st = direct_init(&d, n, op);
    if (st == OR_OK) direct_solve(&d, f, psi);
    direct_free(&d);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid.  Level 0 is the fine grid; a level is halved while its
 * interval count is even and at least 4, so the coarsest level has 2, 3, 5 or
 * 7 intervals (N must be 2^k, 3*2^k, 5*2^k or 7*2^k), where nuc sweeps of the
 * smoother stand in for a solve.  Coarse operators are the same
 * discretisation re-applied with the coarse h. */
#define OR_MAX_LEVELS 16

typedef struct {
    int N;
    double *psi, *f, *r;
} or_level;

/* solver OR_SOLVER_MG: one "cycle" is a V(nu1, nu2) cycle; OR_SOLVER_SOR:
 * one "cycle" is sor_sweeps lexicographic SOR sweeps on the fine grid.
 * ldir: the level solved exactly (reading R15), -1 if none (then the V-cycle
 * goes down to the coarsest level and smooths there). */
#define OR_DIRECT_MAX 16

typedef struct {
    int op, nlev, nu1, nu2, nuc, solver, sor_sweeps, ldir;
    double beta;
    or_level lev[OR_MAX_LEVELS];
    or_direct dir;
} or_mg;

static int mg_level_count(int N) {
    int n = 1;
    while (N % 2 == 0 && N >= 4) {
        N /= 2;
        ++n;
    }
    return (N == 2 || N == 3 || N == 5 || N == 7) ? n : -1;
}

/* Turns the exact coarse solve of reading R15 on or off. */
static int mg_set_direct(or_mg *mg, int on) {
    if (mg->ldir >= 0) direct_free(&mg->dir);
    mg->ldir = -1;
    if (!on) return OR_OK;
    for (int l = 1; l < mg->nlev; ++l)
        if (mg->lev[l].N <= OR_DIRECT_MAX) {
            mg->ldir = l;
            return direct_init(&mg->dir, mg->lev[l].N, mg->op);
        }
    return OR_OK;
}

static int mg_init(or_mg *mg, int N, int op) {
    int nlev = mg_level_count(N);
    if (nlev < 1 || nlev > OR_MAX_LEVELS) return OR_ERR_ARG;
    mg->op = op;
    mg->nlev = nlev;
    mg->nu1 = 2; /* V(2,1), the library's default: the paper fixes no */
    mg->nu2 = 1; /* smoothing counts (reading R7)                      */
    mg->nuc = 16;
    mg->solver = OR_SOLVER_MG;
    mg->sor_sweeps = 16;
    mg->beta = 1.1; /* relaxation of Eq. (15) in the smoother (the library's default) */
    for (int l = 0; l < nlev; ++l) {
        int n = N >> l;
        size_t m = (size_t)(n + 1) * (n + 1);
        mg->lev[l].N = n;
        mg->lev[l].psi = l == 0 ? NULL : calloc(m, sizeof(double));
        mg->lev[l].f = l == 0 ? NULL : calloc(m, sizeof(double));
        mg->lev[l].r = calloc(m, sizeof(double));
    }
    mg->ldir = -1;
    return mg_set_direct(mg, 1);
}

static void mg_free(or_mg *mg) {
    if (mg->ldir >= 0) direct_free(&mg->dir);
    for (int l = 0; l < mg->nlev; ++l) {
        if (l > 0) {
            free(mg->lev[l].psi);
            free(mg->lev[l].f);
        }
        free(mg->lev[l].r);
    }
}

static void vcycle(or_mg *mg, int l) {
    or_level *L = &mg->lev[l];
    if (l == mg->ldir) {
        direct_solve(&mg->dir, L->f, L->psi);
        return;
    }
    if (l == mg->nlev - 1) {
        or_smooth(L->N, mg->op, L->psi, L->f, mg->beta, mg->nuc);
        return;
    }
    or_level *C = &mg->lev[l + 1];
    or_smooth(L->N, mg->op, L->psi, L->f, mg->beta, mg->nu1);
    or_residual(L->N, mg->op, L->psi, L->f, L->r);
    or_restrict(L->N, L->r, C->f);
    memset(C->psi, 0, sizeof(double) * (size_t)(C->N + 1) * (C->N + 1));
    vcycle(mg, l + 1);
    or_prolong_add(C->N, C->psi, L->psi);
    or_smooth(L->N, mg->op, L->psi, L->f, mg->beta, mg->nu2);
}

/* Solve L_h psi = f (reading R7).  psi holds the warm start on entry and the
 * solution on return (walls untouched, i.e. zero).  Returns the number of
 * cycles (V-cycles, or passes of sor_sweeps SOR sweeps); *rel receives
 * ||f - L_h psi|| / ||f|| (0 if both are zero). */
static int mg_solve(or_mg *mg, double *psi, double *f, double tol, int max_cycles, double *rel, int *status) {
    or_level *F = &mg->lev[0];
    F->psi = psi;
    F->f = f;
    double fnorm = interior_norm2(F->N, f);
    int cycles = 0;
    double rnorm;
    for (;;) {
        if (mg->solver == OR_SOLVER_SOR)
            or_sor_lex(F->N, mg->op, psi, f, mg->beta, mg->sor_sweeps);
        else
            vcycle(mg, 0);
        ++cycles;
        or_residual(F->N, mg->op, psi, f, F->r);
        rnorm = interior_norm2(F->N, F->r);
        if (!(rnorm == rnorm) || !(fnorm == fnorm)) {
            *status = OR_ERR_NONFINITE;
            break;
        }
        if (rnorm <= tol * fnorm) break;
        if (cycles >= max_cycles) {
            *status = OR_ERR_NOCONV;
            break;
        }
    }
    *rel = fnorm > 0.0 ? rnorm / fnorm : (rnorm > 0.0 ? INFINITY : 0.0);
    F->psi = NULL;
    F->f = NULL;
    return cycles;
}

/* Stand-alone Poisson solve for the pins: L_h psi = f on an N-interval grid;
 * direct = 1 solves the first level below the finest with at most 16
 * intervals exactly (R15), 0 smooths the coarsest level (R12). */
int or_poisson_solve2(int N, int op, const double *f, double *psi, double tol, int max_cycles, int nu1, int nu2,
                      double beta, int direct, double *rel_out) {
    or_mg mg;
    if (mg_init(&mg, N, op) != OR_OK || mg_set_direct(&mg, direct) != OR_OK) return OR_ERR_ARG;
    mg.nu1 = nu1;
    mg.nu2 = nu2;
    mg.beta = beta;
    size_t m = (size_t)(N + 1) * (N + 1);
    double *fc = malloc(sizeof(double) * m);
    memcpy(fc, f, sizeof(double) * m);
    int status = OR_OK;
    double rel = 0.0;
    int cycles = mg_solve(&mg, psi, fc, tol, max_cycles, &rel, &status);
    if (rel_out) *rel_out = rel;
    free(fc);
    mg_free(&mg);
    return status == OR_OK ? cycles : status;
}

int or_poisson_solve(int N, int op, const double *f, double *psi, double tol, int max_cycles, int nu1, int nu2,
                     double beta, double *rel_out) {
    return or_poisson_solve2(N, op, f, psi, tol, max_cycles, nu1, nu2, beta, 1, rel_out);
}

/* Stand-alone lexicographic SOR solve for the pins: passes of sweeps_per_check
 * sweeps, each followed by the stopping test of mg_solve. */
int or_sor_solve(int N, int op, const double *f, double *psi, double tol, int max_checks, int sweeps_per_check,
                 double beta, double *rel_out) {
    or_mg mg;
    if (mg_init(&mg, N, op) != OR_OK) return OR_ERR_ARG;
    mg.solver = OR_SOLVER_SOR;
    mg.sor_sweeps = sweeps_per_check;
    mg.beta = beta;
    size_t m = (size_t)(N + 1) * (N + 1);
    double *fc = malloc(sizeof(double) * m);
    memcpy(fc, f, sizeof(double) * m);
    int status = OR_OK;
    double rel = 0.0;
    int cycles = mg_solve(&mg, psi, fc, tol, max_checks, &rel, &status);
    if (rel_out) *rel_out = rel;
    free(fc);
    mg_free(&mg);
    return status == OR_OK ? cycles : status;
}

/* ------------------------------------------------------------------------ */
/* Wall vorticity by Thom's method, Eq. (25), reading R2/R3.  The lid speed at
 * node i is U * profile(x_i): profile 0 is the uniform lid of Sec. 3.2, profile
 * 1 the regularised lid 16 x^2 (1 - x)^2 used only by convergence tests. */
static double lid_speed(double U, int profile, double x) {
    if (profile == 1) return U * 16.0 * x * x * (1.0 - x) * (1.0 - x);
    return U;
}

void or_thom(int N, double U, int profile, const double *psi, double *omega) {
    double h = 1.0 / N;
    for (int i = 1; i < N; ++i) {
        omega[AT(N, i, 0)] = -2.0 * psi[AT(N, i, 1)] / (h * h);
        omega[AT(N, i, N)] = -2.0 * psi[AT(N, i, N - 1)] / (h * h) - 2.0 * lid_speed(U, profile, i * h) / h;
    }
    for (int j = 1; j < N; ++j) {
        omega[AT(N, 0, j)] = -2.0 * psi[AT(N, 1, j)] / (h * h);
        omega[AT(N, N, j)] = -2.0 * psi[AT(N, N - 1, j)] / (h * h);
    }
    omega[AT(N, 0, 0)] = omega[AT(N, N, 0)] = omega[AT(N, 0, N)] = omega[AT(N, N, N)] = 0.0;
}

/* L(omega) at interior nodes, Eq. (8), with u and v from Eq. (22) and
 * nu = 1/Re.  advect = 0 drops the two transport terms (Stokes limit tests). */
void or_rhs_L(int N, double Re, int advect, const double *psi, const double *omega, double *out) {
    double h = 1.0 / N, dx = h, dy = h, nu = 1.0 / Re;
    memset(out, 0, sizeof(double) * (size_t)(N + 1) * (N + 1));
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) {
            double u = (psi[AT(N, i, j + 1)] - psi[AT(N, i, j - 1)]) / (2.0 * dy);
            double v = -(psi[AT(N, i + 1, j)] - psi[AT(N, i - 1, j)]) / (2.0 * dx);
            double wP = omega[AT(N, i, j)];
            double wE = omega[AT(N, i + 1, j)], wW = omega[AT(N, i - 1, j)];
            double wN = omega[AT(N, i, j + 1)], wS = omega[AT(N, i, j - 1)];
            double transport = -u * (wE - wW) / (2.0 * dx) - v * (wN - wS) / (2.0 * dy);
            double diffusion = nu * ((wE - 2.0 * wP + wW) / (dx * dx) + (wN - 2.0 * wP + wS) / (dy * dy));
            out[AT(N, i, j)] = (advect ? transport : 0.0) + diffusion;
        }
}

/* Steady-state monitors between two consecutive states, Eqs. (26)-(27):
 * out[0] = max |omega' - omega| / dt, out[1] = RES_psi, out[2] = RES_omega,
 * with the 1/N factor read as 1/(points per side) = 1/(N+1). */
void or_monitors(int N, double dt, const double *psi0, const double *psi1, const double *om0, const double *om1,
                 double *out) {
    double mx = 0.0, sp = 0.0, so = 0.0;
    for (int j = 0; j <= N; ++j)
        for (int i = 0; i <= N; ++i) {
            double dw = fabs(om1[AT(N, i, j)] - om0[AT(N, i, j)]);
            if (dw > mx) mx = dw;
            so += dw;
            sp += fabs(psi1[AT(N, i, j)] - psi0[AT(N, i, j)]);
        }
    out[0] = mx / dt;
    out[1] = sp / (N + 1);
    out[2] = so / (N + 1);
}

/* ------------------------------------------------------------------------ */
/* The cavity: state (psi, omega) and the time step. */
#define OR_MAX_LOG 1000000

typedef struct {
    int N, op, advect, profile, max_cycles;
    double Re, dt, tol, U;
    double *psi, *omega, *f, *L, *y, *work;
    or_mg mg;
    int status;
    double last_rel;
    int last_cycles;
    long long step_count;
    int *cycle_log;
    long long nlog;
} or_cavity;

static size_t nodes(int N) { return (size_t)(N + 1) * (N + 1); }

/* Interior vorticity is the Runge-Kutta unknown; it is packed row by row. */
static void scatter_interior(int N, const double *y, double *omega) {
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) omega[AT(N, i, j)] = y[(size_t)(j - 1) * (N - 1) + (i - 1)];
}

static void gather_interior(int N, const double *field, double *y) {
#pragma omp parallel for schedule(static) num_threads(or_threads) if (or_par(N))
    for (int j = 1; j < N; ++j)
        for (int i = 1; i < N; ++i) y[(size_t)(j - 1) * (N - 1) + (i - 1)] = field[AT(N, i, j)];
}

/* Poisson solve for the current omega (lagged walls, R6), then Thom (R5). */
static void cavity_solve(or_cavity *cv) {
    or_poisson_rhs(cv->N, cv->op, cv->omega, cv->f);
    int st = OR_OK;
    cv->last_cycles = mg_solve(&cv->mg, cv->psi, cv->f, cv->tol, cv->max_cycles, &cv->last_rel, &st);
    if (st != OR_OK && cv->status == OR_OK) cv->status = st;
    if (cv->nlog < OR_MAX_LOG) cv->cycle_log[cv->nlog++] = cv->last_cycles;
    or_thom(cv->N, cv->U, cv->profile, cv->psi, cv->omega);
}

/* L at Runge-Kutta stage input s.  For s = 0 (omega^n) psi is already the
 * solution from the end of the previous step (R8). */
static void cavity_L(void *user, int stage, const double *y, double *out) {
    or_cavity *cv = (or_cavity *)user;
    scatter_interior(cv->N, y, cv->omega);
    if (stage > 0) cavity_solve(cv);
    or_rhs_L(cv->N, cv->Re, cv->advect, cv->psi, cv->omega, cv->L);
    gather_interior(cv->N, cv->L, out);
}

void *or_create(int N, double Re, double dt, double tol, int op) {
    if (mg_level_count(N) < 2 || Re <= 0.0 || dt <= 0.0 || tol <= 0.0 || (op != OR_OP_5PT && op != OR_OP_COMPACT))
        return NULL;
    or_cavity *cv = calloc(1, sizeof(or_cavity));
    cv->N = N;
    cv->op = op;
    cv->Re = Re;
    cv->dt = dt;
    cv->tol = tol;
    cv->U = 1.0;
    cv->advect = 1;
    cv->profile = 0;
    cv->max_cycles = 100;
    size_t m = nodes(N), ni = (size_t)(N - 1) * (N - 1);
    cv->psi = calloc(m, sizeof(double));
    cv->omega = calloc(m, sizeof(double));
    cv->f = calloc(m, sizeof(double));
    cv->L = calloc(m, sizeof(double));
    cv->y = calloc(ni, sizeof(double));
    cv->work = calloc(11 * ni, sizeof(double));
    cv->cycle_log = calloc(OR_MAX_LOG, sizeof(int));
    mg_init(&cv->mg, N, op);
    /* Start from rest: omega = 0 gives f = 0 and psi = 0; Thom then puts the
     * lid's -2U/h on the top wall. */
    or_thom(N, cv->U, cv->profile, cv->psi, cv->omega);
    return cv;
}

void or_destroy(void *p) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv) return;
    mg_free(&cv->mg);
    free(cv->psi);
    free(cv->omega);
    free(cv->f);
    free(cv->L);
    free(cv->y);
    free(cv->work);
    free(cv->cycle_log);
    free(cv);
}

/* Options: "U", "profile", "advect", "max_cycles", "nu1", "nu2", "nuc",
 * "beta", "solver" (0 multigrid, 1 lexicographic SOR), "sor_sweeps",
 * "coarse_direct" (1 default: reading R15; 0: reading R12).
 * Changing the lid re-applies Thom to the current psi. */
int or_set_option(void *p, const char *key, double value) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv || !key) return OR_ERR_ARG;
    if (!strcmp(key, "U") || !strcmp(key, "profile")) {
        if (!strcmp(key, "U")) cv->U = value;
        else cv->profile = (int)value;
        or_thom(cv->N, cv->U, cv->profile, cv->psi, cv->omega);
    } else if (!strcmp(key, "advect")) cv->advect = (int)value;
    else if (!strcmp(key, "max_cycles")) cv->max_cycles = (int)value;
    else if (!strcmp(key, "nu1")) cv->mg.nu1 = (int)value;
    else if (!strcmp(key, "nu2")) cv->mg.nu2 = (int)value;
    else if (!strcmp(key, "nuc")) cv->mg.nuc = (int)value;
    else if (!strcmp(key, "beta")) cv->mg.beta = value;
    else if (!strcmp(key, "solver")) cv->mg.solver = (int)value;
    else if (!strcmp(key, "sor_sweeps")) cv->mg.sor_sweeps = (int)value;
    else if (!strcmp(key, "coarse_direct")) return mg_set_direct(&cv->mg, (int)value);
    else return OR_ERR_ARG;
    return OR_OK;
}

/* nsteps SSPRK(5,4) steps.  Returns OR_OK or the first error seen. */
int or_step(void *p, int nsteps) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv || nsteps < 0) return OR_ERR_ARG;
    int N = cv->N;
    for (int s = 0; s < nsteps; ++s) {
        gather_interior(N, cv->omega, cv->y);
        or_ssprk54_step((N - 1) * (N - 1), cv->y, cv->dt, cavity_L, cv, cv->work);
        scatter_interior(N, cv->y, cv->omega);
        cavity_solve(cv);
        cv->step_count++;
    }
    return cv->status;
}

/* field 0 = psi, 1 = omega; (N+1)^2 values, index j*(N+1)+i. */
int or_get(void *p, int field, double *out) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv || field < 0 || field > 1) return OR_ERR_ARG;
    memcpy(out, field == 0 ? cv->psi : cv->omega, sizeof(double) * nodes(cv->N));
    return OR_OK;
}

/* Installs a state.  psi is taken as given; omega's interior is taken and its
 * walls are recomputed from psi by Thom, so the pair is the state the end of a
 * step would leave. */
int or_set_state(void *p, const double *psi, const double *omega) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv) return OR_ERR_ARG;
    memcpy(cv->psi, psi, sizeof(double) * nodes(cv->N));
    memcpy(cv->omega, omega, sizeof(double) * nodes(cv->N));
    or_thom(cv->N, cv->U, cv->profile, cv->psi, cv->omega);
    return OR_OK;
}

double or_last_residual(void *p) { return p ? ((or_cavity *)p)->last_rel : NAN; }

/* Copies up to max cycle counts (one per Poisson solve, oldest first). */
long long or_cycle_log(void *p, int *out, long long max) {
    or_cavity *cv = (or_cavity *)p;
    if (!cv) return OR_ERR_ARG;
    long long n = cv->nlog < max ? cv->nlog : max;
    memcpy(out, cv->cycle_log, sizeof(int) * (size_t)n);
    return n;
}
