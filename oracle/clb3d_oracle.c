/*
 * clb3d_oracle.c -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, slow FP64 CPU implementation of the three-dimensional form of the coupled
 * central-moment lattice Boltzmann method of Fei, Luo, Lin & Li (arXiv:1710.10569). The paper
 * gives the method in two dimensions (D2Q9 flow, Sec. 2.1, Eqs. 4-13; D2Q5 temperature, Sec. 2.2,
 * Eqs. 14-23) and states in its conclusions that it extends to three dimensions directly. This file
 * is that extension, built by applying the paper's definitions on the 3-D lattices:
 *   - D3Q27 flow populations (velocities e in {0, +1, -1}^3). Raw moments k_abc = sum_i
 *     e_x^a e_y^b e_z^c f_i with a, b, c in {0, 1, 2} (the 3-D analogue of Eq. 7a); central moments
 *     k~_abc = sum_i (e_x-u_x)^a (e_y-u_y)^b (e_z-u_z)^c f_i (Eq. 5), whose shift matrix N(u) is
 *     written out here from the binomial expansion of that definition.
 *   - Equilibrium central moments of the continuous Maxwellian restricted to the lattice, as Eq. 9:
 *     k~eq_abc = rho * m(a) m(b) m(c) with m(0) = 1, m(1) = 0, m(2) = cs2.
 *   - Forcing central moments, as Eq. 11: C_abc = F_d * prod_{d' != d} m(a_d') when exactly one
 *     index a_d equals 1, else 0 (in 2-D this gives C = [0, Fx, Fy, 0, 0, 0, cs2 Fy, cs2 Fx, 0]).
 *   - Relaxation, as Eq. 8: Gamma~* = Gamma~ - S (Gamma~ - Gamma~eq) + (I - S/2) C with S zero on the
 *     conserved moments, s_nu on k~110, k~101, k~011, on the three normal second moments the
 *     block s_nu I + (s_b - s_nu)/3 J (their trace relaxes with s_b, their deviators with s_nu; in
 *     2-D the same rule gives the paper's s+/s- block), s_3 on third-order, s_4 on fourth-order,
 *     s_5 on fifth-order and s_6 on the sixth-order moment.
 *   - D3Q7 temperature populations, moments 1, e_x, e_y, e_z, e_x^2, e_y^2, e_z^2 (the analogue of
 *     Eq. 17), central moments about the flow velocity (Eq. 18 written out from the definition),
 *     equilibrium [T, 0, 0, 0, cs2_T T, cs2_T T, cs2_T T] (Eq. 20), relaxation
 *     diag(lambda0, lambda1 x3, lambda2 x3) (Eq. 19).
 *   - Boussinesq force along +axis g_axis: F = Fv + rho0 g_beta (T - T0) e_g (Eq. 3); u = (sum f e +
 *     F/2) / rho with the local rho (Eq. 13); T = sum g (Eq. 23).
 *   - Walls halfway between nodes on any face: f bounces back; g anti-bounces back,
 *     g_i = -g*_opp + 2 w^T_i T_w, on Dirichlet faces and bounces back on adiabatic faces. A wall
 *     face may move with velocity u_w (tangential motion and normal injection alike): then
 *     f_i = f*_opp + [f^eq_i - f^eq_opp](rho0, u_w) and, on Dirichlet faces,
 *     g_i = -g*_opp + [g^eq_i + g^eq_opp](T_w, u_w) (the 2-D moving-wall rule on each face); a
 *     diagonal that crosses several faces at an edge or corner takes the velocity of the face of the
 *     highest axis (z before y before x).
 * M^-1 and M_T^-1 are computed numerically (Gauss-Jordan); N^-1 is applied by solving the unit
 * lower-triangular system. Nothing is fused or reordered: collide every node, then stream.
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg load this file.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * With thermal_only set only the D3Q7 equation is stepped, with the velocity given to orc3_init
 * held fixed (the 3-D form of the Sec. 3.1 set-up).
 *
 * Pins (tests/test_oracle3d_pins.py): moments against brute-force sums, N(u) N(-u) = I,
 * conservation, the equilibrium as a fixed point, a field uniform along one axis reproducing the
 * two-dimensional oracle step for step (all three axis orientations), axis permutation symmetry,
 * the decay rate of a 3-D shear wave, body-force Poiseuille flow between walls and steady
 * conduction between Dirichlet walls.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define Q27 27
#define Q7 7
#define ORC3_OMP_MIN_NODES 1024

enum { ORC3_PERIODIC = 0, ORC3_DIRICHLET = 1, ORC3_ADIABATIC = 2 };

typedef struct {
    int nx, ny, nz;
    double nu, kappa, g_beta, T0, rho0;
    double s_b, s_3, s_4, s_5, s_6, lambda0, lambda2, cs2_T;
    double Fv[3];
    int g_axis;       /* buoyancy acts along +g_axis (0: x, 1: y, 2: z) */
    int wall[6];      /* faces -x, +x, -y, +y, -z, +z */
    double T_wall[6];
    double u_wall[6][3]; /* velocity of each wall face */
    int thermal_only;    /* 1: only the D3Q7 equation, with the velocity given to orc3_init held fixed */
} orc3_params;

/* Velocity component of index digit 0, 1, 2: 0, +1, -1. Population i has digits (i%3, i/3%3, i/9). */
static int digit_vel(int d) { return d == 0 ? 0 : (d == 1 ? 1 : -1); }
static int ex27(int i) { return digit_vel(i % 3); }
static int ey27(int i) { return digit_vel((i / 3) % 3); }
static int ez27(int i) { return digit_vel(i / 9); }

/* D3Q7: rest, +x, -x, +y, -y, +z, -z. */
static const int EX7[Q7] = {0, 1, -1, 0, 0, 0, 0};
static const int EY7[Q7] = {0, 0, 0, 1, -1, 0, 0};
static const int EZ7[Q7] = {0, 0, 0, 0, 0, 1, -1};

typedef struct {
    orc3_params p;
    double cs2, s_nu, lambda1;
    double M[Q27][Q27], Minv[Q27][Q27], S[Q27][Q27];
    double MT[Q7][Q7], MTinv[Q7][Q7], ST[Q7][Q7];
    int opp[Q27], oppT[Q7];
    double wT[Q7];
    double fwall[6][Q27];   /* f^eq(rho0, u_wall) of each face */
    double gwall[6][Q7];    /* g^eq(T_wall, u_wall) of each face */
    double *f, *g, *fs, *gs; /* [q][z][y][x] */
    double *up[3];           /* prescribed velocity of the thermal-only mode, [z][y][x] */
    long steps;
} orc3_sim;

static double ipow(double x, int n)
{
    double r = 1.0;
    for (int k = 0; k < n; ++k) r *= x;
    return r;
}

static double binom(int n, int k)
{
    double r = 1.0;
    for (int j = 1; j <= k; ++j) r = r * (n - k + j) / j;
    return r;
}

/* ---------------------------------------------------------------- moment matrices */

/* Moment m has exponents (m%3, m/3%3, m/9) on (e_x, e_y, e_z). */
static void build_M(double M[Q27][Q27])
{
    for (int m = 0; m < Q27; ++m)
        for (int i = 0; i < Q27; ++i)
            M[m][i] = ipow(ex27(i), m % 3) * ipow(ey27(i), (m / 3) % 3) * ipow(ez27(i), m / 9);
}

/* Central moment k~_abc = sum_{a'<=a, b'<=b, c'<=c} C(a,a') C(b,b') C(c,c') (-u_x)^(a-a')
 * (-u_y)^(b-b') (-u_z)^(c-c') k_a'b'c', from expanding (e-u)^a per axis. */
static void build_N(double ux, double uy, double uz, double N[Q27][Q27])
{
    const double u[3] = {ux, uy, uz};
    for (int m = 0; m < Q27; ++m) {
        const int a[3] = {m % 3, (m / 3) % 3, m / 9};
        for (int n = 0; n < Q27; ++n) {
            const int b[3] = {n % 3, (n / 3) % 3, n / 9};
            double v = 1.0;
            for (int d = 0; d < 3; ++d) {
                if (b[d] > a[d]) { v = 0.0; break; }
                v *= binom(a[d], b[d]) * ipow(-u[d], a[d] - b[d]);
            }
            N[m][n] = v;
        }
    }
}

/* D3Q7 moments 1, e_x, e_y, e_z, e_x^2, e_y^2, e_z^2. */
static void build_MT(double M[Q7][Q7])
{
    for (int i = 0; i < Q7; ++i) {
        M[0][i] = 1.0;
        M[1][i] = EX7[i];
        M[2][i] = EY7[i];
        M[3][i] = EZ7[i];
        M[4][i] = EX7[i] * EX7[i];
        M[5][i] = EY7[i] * EY7[i];
        M[6][i] = EZ7[i] * EZ7[i];
    }
}

/* k~_d = k_d - u_d T, k~_dd = k_dd - 2 u_d k_d + u_d^2 T. */
static void build_NT(double ux, double uy, double uz, double N[Q7][Q7])
{
    const double u[3] = {ux, uy, uz};
    memset(N, 0, sizeof(double) * Q7 * Q7);
    N[0][0] = 1.0;
    for (int d = 0; d < 3; ++d) {
        N[1 + d][0] = -u[d];
        N[1 + d][1 + d] = 1.0;
        N[4 + d][0] = u[d] * u[d];
        N[4 + d][1 + d] = -2.0 * u[d];
        N[4 + d][4 + d] = 1.0;
    }
}

/* ---------------------------------------------------------------- plain linear algebra */

static int invert(int n, const double *A, double *Ainv)
{
    double *a = (double *)malloc(sizeof(double) * n * 2 * n);
    if (!a) return -1;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c) a[r * 2 * n + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * 2 * n + c]) > fabs(a[piv * 2 * n + c])) piv = r;
        if (a[piv * 2 * n + c] == 0.0) { free(a); return -1; }
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) {
                const double t = a[c * 2 * n + k];
                a[c * 2 * n + k] = a[piv * 2 * n + k];
                a[piv * 2 * n + k] = t;
            }
        const double d = a[c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) a[c * 2 * n + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double fct = a[r * 2 * n + c];
            if (fct == 0.0) continue;
            for (int k = 0; k < 2 * n; ++k) a[r * 2 * n + k] -= fct * a[c * 2 * n + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * 2 * n + n + c];
    free(a);
    return 0;
}

static void matvec(int n, const double *A, const double *x, double *y)
{
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += A[r * n + c] * x[c];
        y[r] = s;
    }
}

static void solve_unit_lower(int n, const double *L, const double *b, double *x)
{
    for (int r = 0; r < n; ++r) {
        double s = b[r];
        for (int c = 0; c < r; ++c) s -= L[r * n + c] * x[c];
        x[r] = s;
    }
}

/* ---------------------------------------------------------------- set-up */

static int order_of(int m) { return m % 3 + (m / 3) % 3 + m / 9; }

static void build_constants(orc3_sim *s)
{
    const orc3_params *p = &s->p;
    s->cs2 = 1.0 / 3.0;
    s->s_nu = 1.0 / (p->nu / s->cs2 + 0.5);
    s->lambda1 = 1.0 / (p->kappa / p->cs2_T + 0.5);
    build_M(s->M);
    invert(Q27, &s->M[0][0], &s->Minv[0][0]);
    build_MT(s->MT);
    invert(Q7, &s->MT[0][0], &s->MTinv[0][0]);

    memset(s->S, 0, sizeof(s->S));
    const int normal2[3] = {2, 6, 18}; /* (2,0,0), (0,2,0), (0,0,2) */
    for (int m = 0; m < Q27; ++m) {
        const int o = order_of(m);
        double r = 0.0;
        if (o == 2) r = s->s_nu; /* off-diagonal second moments; the normal ones are set below */
        if (o == 3) r = p->s_3;
        if (o == 4) r = p->s_4;
        if (o == 5) r = p->s_5;
        if (o == 6) r = p->s_6;
        s->S[m][m] = r;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            s->S[normal2[i]][normal2[j]] = (i == j ? s->s_nu : 0.0) + (p->s_b - s->s_nu) / 3.0;

    memset(s->ST, 0, sizeof(s->ST));
    s->ST[0][0] = p->lambda0;
    for (int d = 0; d < 3; ++d) {
        s->ST[1 + d][1 + d] = s->lambda1;
        s->ST[4 + d][4 + d] = p->lambda2;
    }
    for (int i = 0; i < Q27; ++i)
        for (int j = 0; j < Q27; ++j)
            if (ex27(j) == -ex27(i) && ey27(j) == -ey27(i) && ez27(j) == -ez27(i)) s->opp[i] = j;
    for (int i = 0; i < Q7; ++i)
        for (int j = 0; j < Q7; ++j)
            if (EX7[j] == -EX7[i] && EY7[j] == -EY7[i] && EZ7[j] == -EZ7[i]) s->oppT[i] = j;
    const double geq[Q7] = {1.0, 0.0, 0.0, 0.0, p->cs2_T, p->cs2_T, p->cs2_T};
    matvec(Q7, &s->MTinv[0][0], geq, s->wT);
}

/* m(0) = 1, m(1) = 0, m(2) = cs2: the 1-D central moments of the lattice Maxwellian. */
static double mw(int a, double cs2) { return a == 0 ? 1.0 : (a == 1 ? 0.0 : cs2); }

static void eq_moments(double rho, double cs2, double geq[Q27])
{
    for (int m = 0; m < Q27; ++m) geq[m] = rho * mw(m % 3, cs2) * mw((m / 3) % 3, cs2) * mw(m / 9, cs2);
}

static void force_moments(const double F[3], double cs2, double C[Q27])
{
    for (int m = 0; m < Q27; ++m) {
        const int a[3] = {m % 3, (m / 3) % 3, m / 9};
        double c = 0.0;
        for (int d = 0; d < 3; ++d) {
            if (a[d] != 1) continue;
            double prod = F[d];
            for (int e = 0; e < 3; ++e)
                if (e != d) prod *= mw(a[e], cs2); /* zero when another index is 1 */
            c += prod;
        }
        C[m] = c;
    }
}

/* ---------------------------------------------------------------- one node */

static void macroscopic(const orc3_sim *s, const double f[Q27], const double g[Q7], double *rho,
                        double u[3], double *T, double F[3])
{
    const orc3_params *p = &s->p;
    double r = 0.0, j[3] = {0, 0, 0}, t = 0.0;
    for (int i = 0; i < Q27; ++i) {
        r += f[i];
        j[0] += f[i] * ex27(i);
        j[1] += f[i] * ey27(i);
        j[2] += f[i] * ez27(i);
    }
    for (int i = 0; i < Q7; ++i) t += g[i];
    for (int d = 0; d < 3; ++d) F[d] = p->Fv[d];
    F[p->g_axis] += p->rho0 * p->g_beta * (t - p->T0);
    *rho = r;
    *T = t;
    for (int d = 0; d < 3; ++d) u[d] = (j[d] + 0.5 * F[d]) / r;
}

/* D3Q7 collision (Eqs. 16-21 in 3-D) with the velocity u; T = sum g. */
static void collide_d3q7(const orc3_sim *s, const double g[Q7], const double u[3], double go[Q7])
{
    double T = 0.0;
    for (int i = 0; i < Q7; ++i) T += g[i];
    double NT[Q7][Q7], gamT[Q7], gtT[Q7], dT[Q7], SdT[Q7], gtsT[Q7], gamsT[Q7];
    build_NT(u[0], u[1], u[2], NT);
    matvec(Q7, &s->MT[0][0], g, gamT);
    matvec(Q7, &NT[0][0], gamT, gtT);
    const double c2 = s->p.cs2_T;
    const double geqT[Q7] = {T, 0, 0, 0, T * c2, T * c2, T * c2};
    for (int k = 0; k < Q7; ++k) dT[k] = gtT[k] - geqT[k];
    matvec(Q7, &s->ST[0][0], dT, SdT);
    for (int k = 0; k < Q7; ++k) gtsT[k] = gtT[k] - SdT[k];
    solve_unit_lower(Q7, &NT[0][0], gtsT, gamsT);
    matvec(Q7, &s->MTinv[0][0], gamsT, go);
}

static void collide(const orc3_sim *s, const double f[Q27], const double g[Q7], double fo[Q27],
                    double go[Q7])
{
    const orc3_params *p = &s->p;
    double rho, u[3], T, F[3];
    macroscopic(s, f, g, &rho, u, &T, F);

    /* ---- D3Q27 ---- */
    double Nl[Q27][Q27];
    build_N(u[0], u[1], u[2], Nl);
    double gam[Q27], gt[Q27], geq[Q27], C[Q27], d[Q27], Sd[Q27], SC[Q27], gts[Q27], gams[Q27];
    matvec(Q27, &s->M[0][0], f, gam);
    matvec(Q27, &Nl[0][0], gam, gt);
    eq_moments(rho, s->cs2, geq);
    force_moments(F, s->cs2, C);
    for (int k = 0; k < Q27; ++k) d[k] = gt[k] - geq[k];
    matvec(Q27, &s->S[0][0], d, Sd);
    matvec(Q27, &s->S[0][0], C, SC);
    for (int k = 0; k < Q27; ++k) gts[k] = gt[k] - Sd[k] + C[k] - 0.5 * SC[k];
    solve_unit_lower(Q27, &Nl[0][0], gts, gams);
    matvec(Q27, &s->Minv[0][0], gams, fo);

    collide_d3q7(s, g, u, go);
}

static void equilibrium(const orc3_sim *s, double rho, const double u[3], double T, double f[Q27],
                        double g[Q7])
{
    double N[Q27][Q27], NT[Q7][Q7], geq[Q27], gam[Q27], gamT[Q7];
    build_N(u[0], u[1], u[2], N);
    eq_moments(rho, s->cs2, geq);
    solve_unit_lower(Q27, &N[0][0], geq, gam);
    matvec(Q27, &s->Minv[0][0], gam, f);
    const double c2 = s->p.cs2_T;
    const double geqT[Q7] = {T, 0, 0, 0, T * c2, T * c2, T * c2};
    build_NT(u[0], u[1], u[2], NT);
    solve_unit_lower(Q7, &NT[0][0], geqT, gamT);
    matvec(Q7, &s->MTinv[0][0], gamT, g);
}

/* ---------------------------------------------------------------- lattice */

static size_t nodes(const orc3_sim *s) { return (size_t)s->p.nx * s->p.ny * s->p.nz; }

/* Pull streaming: population i at x comes from x - e_i; a pull across a wall face takes the
 * node's own post-collision opposite population (for g with the anti-bounce-back term on a
 * Dirichlet face). A diagonal that crosses two or three faces bounces back the same way. */
static void stream(orc3_sim *s)
{
    const orc3_params *p = &s->p;
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t n = nodes(s);
#pragma omp parallel for collapse(2) schedule(static) if (n >= ORC3_OMP_MIN_NODES)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const size_t here = ((size_t)z * ny + y) * nx + x;
                for (int i = 0; i < Q27; ++i) {
                    int c[3] = {x - ex27(i), y - ey27(i), z - ez27(i)};
                    const int len[3] = {nx, ny, nz};
                    int face = -1; /* the face crossed; of several, that of the highest axis */
                    for (int d = 0; d < 3; ++d) {
                        if (c[d] < 0) {
                            if (p->wall[2 * d] == ORC3_PERIODIC) c[d] += len[d]; else face = 2 * d;
                        } else if (c[d] >= len[d]) {
                            if (p->wall[2 * d + 1] == ORC3_PERIODIC) c[d] -= len[d]; else face = 2 * d + 1;
                        }
                    }
                    const int o = s->opp[i];
                    if (face < 0)
                        s->f[i * n + here] = s->fs[i * n + ((size_t)c[2] * ny + c[1]) * nx + c[0]];
                    else
                        s->f[i * n + here] = s->fs[o * n + here] + (s->fwall[face][i] - s->fwall[face][o]);
                }
                for (int i = 0; i < Q7; ++i) {
                    int c[3] = {x - EX7[i], y - EY7[i], z - EZ7[i]};
                    const int len[3] = {nx, ny, nz};
                    int face = -1;
                    for (int d = 0; d < 3; ++d) {
                        if (c[d] < 0) {
                            if (p->wall[2 * d] == ORC3_PERIODIC) c[d] += len[d]; else face = 2 * d;
                        } else if (c[d] >= len[d]) {
                            if (p->wall[2 * d + 1] == ORC3_PERIODIC) c[d] -= len[d]; else face = 2 * d + 1;
                        }
                    }
                    const int o = s->oppT[i];
                    if (face < 0)
                        s->g[i * n + here] = s->gs[i * n + ((size_t)c[2] * ny + c[1]) * nx + c[0]];
                    else if (p->wall[face] == ORC3_DIRICHLET)
                        s->g[i * n + here] = -s->gs[o * n + here] + (s->gwall[face][i] + s->gwall[face][o]);
                    else
                        s->g[i * n + here] = s->gs[o * n + here];
                }
            }
}

static void collide_all(orc3_sim *s)
{
    const long n = (long)nodes(s);
#pragma omp parallel for schedule(static) if (n >= ORC3_OMP_MIN_NODES)
    for (long k = 0; k < n; ++k) {
        double f[Q27], g[Q7], fo[Q27], go[Q7];
        for (int i = 0; i < Q27; ++i) f[i] = s->f[i * n + k];
        for (int i = 0; i < Q7; ++i) g[i] = s->g[i * n + k];
        if (s->p.thermal_only) {
            const double u[3] = {s->up[0][k], s->up[1][k], s->up[2][k]};
            for (int i = 0; i < Q27; ++i) fo[i] = f[i];
            collide_d3q7(s, g, u, go);
        } else {
            collide(s, f, g, fo, go);
        }
        for (int i = 0; i < Q27; ++i) s->fs[i * n + k] = fo[i];
        for (int i = 0; i < Q7; ++i) s->gs[i * n + k] = go[i];
    }
}

/* ---------------------------------------------------------------- exported API (ctypes) */

int orc3_create(const orc3_params *p, orc3_sim **out)
{
    *out = NULL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1 || p->g_axis < 0 || p->g_axis > 2) return -1;
    for (int d = 0; d < 3; ++d)
        if ((p->wall[2 * d] == ORC3_PERIODIC) != (p->wall[2 * d + 1] == ORC3_PERIODIC)) return -1;
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return -2;
    s->p = *p;
    build_constants(s);
    for (int face = 0; face < 6; ++face)
        equilibrium(s, p->rho0, p->u_wall[face], p->T_wall[face], s->fwall[face], s->gwall[face]);
    const size_t n = nodes(s);
    s->f = (double *)calloc(Q27 * n, sizeof(double));
    s->fs = (double *)calloc(Q27 * n, sizeof(double));
    s->g = (double *)calloc(Q7 * n, sizeof(double));
    s->gs = (double *)calloc(Q7 * n, sizeof(double));
    for (int d = 0; d < 3; ++d) s->up[d] = (double *)calloc(n, sizeof(double));
    if (!s->f || !s->fs || !s->g || !s->gs || !s->up[0] || !s->up[1] || !s->up[2]) {
        free(s->f); free(s->fs); free(s->g); free(s->gs);
        for (int d = 0; d < 3; ++d) free(s->up[d]);
        free(s);
        return -2;
    }
    *out = s;
    return 0;
}

void orc3_destroy(orc3_sim *s)
{
    if (!s) return;
    free(s->f); free(s->fs); free(s->g); free(s->gs);
    for (int d = 0; d < 3; ++d) free(s->up[d]);
    free(s);
}

/* f = f^eq(rho, u), g = g^eq(T, u) from [nz][ny][nx] fields (in the thermal-only mode u is also
 * kept as the prescribed velocity). */
void orc3_init(orc3_sim *s, const double *rho, const double *ux, const double *uy, const double *uz,
               const double *T)
{
    const size_t n = nodes(s);
    if (s->p.thermal_only) {
        memcpy(s->up[0], ux, n * sizeof(double));
        memcpy(s->up[1], uy, n * sizeof(double));
        memcpy(s->up[2], uz, n * sizeof(double));
    }
    for (size_t k = 0; k < n; ++k) {
        double f[Q27], g[Q7];
        const double u[3] = {ux[k], uy[k], uz[k]};
        equilibrium(s, rho[k], u, T[k], f, g);
        for (int i = 0; i < Q27; ++i) s->f[i * n + k] = f[i];
        for (int i = 0; i < Q7; ++i) s->g[i * n + k] = g[i];
    }
    s->steps = 0;
}

void orc3_step(orc3_sim *s, long nsteps)
{
    for (long t = 0; t < nsteps; ++t) {
        collide_all(s);
        stream(s);
        s->steps++;
    }
}

void orc3_fields(const orc3_sim *s, double *rho, double *ux, double *uy, double *uz, double *T)
{
    const size_t n = nodes(s);
    for (size_t k = 0; k < n; ++k) {
        double f[Q27], g[Q7], u[3], F[3];
        for (int i = 0; i < Q27; ++i) f[i] = s->f[i * n + k];
        for (int i = 0; i < Q7; ++i) g[i] = s->g[i * n + k];
        macroscopic(s, f, g, &rho[k], u, &T[k], F);
        if (s->p.thermal_only)
            for (int d = 0; d < 3; ++d) u[d] = s->up[d][k];
        ux[k] = u[0];
        uy[k] = u[1];
        uz[k] = u[2];
    }
}

void orc3_get_pops(const orc3_sim *s, double *f, double *g)
{
    const size_t n = nodes(s);
    memcpy(f, s->f, Q27 * n * sizeof(double));
    memcpy(g, s->g, Q7 * n * sizeof(double));
}

void orc3_set_pops(orc3_sim *s, const double *f, const double *g)
{
    const size_t n = nodes(s);
    memcpy(s->f, f, Q27 * n * sizeof(double));
    memcpy(s->g, g, Q7 * n * sizeof(double));
}

int orc3_collide_node(const orc3_params *p, const double *f, const double *g, double *fo, double *go)
{
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return -2;
    s->p = *p;
    build_constants(s);
    collide(s, f, g, fo, go);
    free(s);
    return 0;
}

int orc3_equilibrium_node(const orc3_params *p, double rho, double ux, double uy, double uz, double T,
                          double *f, double *g)
{
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return -2;
    s->p = *p;
    build_constants(s);
    const double u[3] = {ux, uy, uz};
    equilibrium(s, rho, u, T, f, g);
    free(s);
    return 0;
}

/* M, M^-1, N(u), S (27 x 27), M_T, M_T^-1, N_T(u), S_T (7 x 7), the D3Q7 rest weights and the
 * velocity sets (27 x 3 and 7 x 3 integers), as the oracle uses them. */
void orc3_matrices(const orc3_params *p, double ux, double uy, double uz, double *M, double *Minv,
                   double *N, double *S, double *MT, double *MTinv, double *NT, double *ST, double *wT,
                   int *e27, int *e7)
{
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return;
    s->p = *p;
    build_constants(s);
    double Nl[Q27][Q27], NTl[Q7][Q7];
    build_N(ux, uy, uz, Nl);
    build_NT(ux, uy, uz, NTl);
    memcpy(M, s->M, sizeof(s->M));
    memcpy(Minv, s->Minv, sizeof(s->Minv));
    memcpy(N, Nl, sizeof(Nl));
    memcpy(S, s->S, sizeof(s->S));
    memcpy(MT, s->MT, sizeof(s->MT));
    memcpy(MTinv, s->MTinv, sizeof(s->MTinv));
    memcpy(NT, NTl, sizeof(NTl));
    memcpy(ST, s->ST, sizeof(s->ST));
    memcpy(wT, s->wT, sizeof(s->wT));
    for (int i = 0; i < Q27; ++i) {
        e27[3 * i] = ex27(i);
        e27[3 * i + 1] = ey27(i);
        e27[3 * i + 2] = ez27(i);
    }
    for (int i = 0; i < Q7; ++i) {
        e7[3 * i] = EX7[i];
        e7[3 * i + 1] = EY7[i];
        e7[3 * i + 2] = EZ7[i];
    }
    free(s);
}

/* D3Q7 collision of one node with a prescribed velocity (the thermal-only mode). */
int orc3_collide_thermal_node(const orc3_params *p, const double *g, double ux, double uy, double uz, double *go)
{
    orc3_sim *s = (orc3_sim *)calloc(1, sizeof(orc3_sim));
    if (!s) return -2;
    s->p = *p;
    build_constants(s);
    const double u[3] = {ux, uy, uz};
    collide_d3q7(s, g, u, go);
    free(s);
    return 0;
}
