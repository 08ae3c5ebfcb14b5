/*
 * clb_oracle.c -- TEST INFRASTRUCTURE, NOT PRODUCT CODE.
 *
 * A plain, slow, obviously-correct FP64 CPU implementation of the coupled central-moment lattice
 * Boltzmann method of Fei, Luo, Lin & Li, "Modeling incompressible thermal flows using a
 * central-moment-based lattice Boltzmann method" (arXiv:1710.10569):
 *   - D2Q9 flow CLB, Sec. 2.1, Eqs. (4)-(13);
 *   - D2Q5 temperature CLB, Sec. 2.2, Eqs. (14)-(23) and Appendix A;
 *   - Boussinesq force, Eq. (3).
 * Every transform is a literal matrix-vector product with the matrices printed in the paper
 * (Eq. 7a, Eq. 7b, Eq. 17, Eq. 18). M^-1 and M_T^-1 are computed numerically (Gauss-Jordan);
 * N^-1 and N_T^-1 are applied by solving the unit lower-triangular system N x = y.
 * Nothing is fused, blocked or reordered: collide every node, then stream every population.
 *
 * Only the test-suite, the package smoke check and the benchmark's CPU-baseline leg load this file.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Readings taken where the paper is silent or garbled (each is also listed in the design notes):
 *   r1  Eq. 7b prints +2u_y in the k~02 row (column k01). Expanding Eq. 5b, (e_y-u_y)^2 =
 *       e_y^2 - 2u_y e_y + u_y^2, so the entry is -2u_y (it is -2u_y in N_T, Eq. 18). Used here.
 *   r4  F is a force density (it enters rho*u in Eq. 13): F = (Fv_x, Fv_y + rho0*g_beta*(T - T0)),
 *       gravity along -y (Eq. 3), g_beta = |g|*beta >= 0.
 *   r6  The velocity that shifts the D2Q5 moments is the force-corrected u of Eq. 13, same node/step.
 *   r7  u = (sum f e + F/2) / rho with the local rho.
 *   r10 Walls (stationary, halfway between nodes): f uses halfway bounce-back on every wall; g uses
 *       anti-bounce-back g_i = -g*_opp + 2 w^T_i T_w on Dirichlet walls and bounce-back g_i = g*_opp
 *       on adiabatic walls. w^T_i are the D2Q5 rest weights (g^eq at T=1, u=0).
 *   r19 Wet walls (ORC_WET, the paper's own conditions, Sec. 3 first paragraph): the wall row of
 *       nodes lies on the wall (r26: x sides alike, the roles of x and y exchanged). After
 *       streaming, the populations that would come from beyond the wall are set by
 *       non-equilibrium bounce-back, f_i = f_opp +
 *       [f^eq_i - f^eq_opp](rho, u'), with u' = u_w - F/(2 rho) so that the force-corrected velocity
 *       of Eq. (13) equals the wall's, rho from mass and normal momentum, and the tangential
 *       momentum closed on the two diagonals; g at the wall node is set by non-equilibrium
 *       extrapolation from the adjacent fluid node n, g_i = g^eq_i(T_w, u_w) + [g_i(n) -
 *       g^eq_i(T(n), u(n))].
 *   r26 Corners of wet walls (a node on an x wall and a y wall): the y wall's velocity and the mean
 *       of the two walls' temperatures; rho from the diagonal fluid neighbour; the unknowns whose
 *       opposite is known by non-equilibrium bounce-back, the two buried diagonals sharing the
 *       remaining mass equally; g by non-equilibrium extrapolation from the diagonal neighbour.
 *       In the thermal-only mode wet walls set g only, with the node's prescribed velocity.
 * Parity is pinned by the tests in tests/test_oracle_pins.py (transform brute force, fixed point,
 * conservation, viscosity and diffusivity decay, Poiseuille, conduction, Table 1 Nusselt numbers).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define Q9 9
#define Q5 5
#define ORC_OMP_MIN_NODES 1024 /* smaller lattices run on one thread */

/* D2Q9 velocity set, Eq. (4). D2Q5 uses the first five (Sec. 2.2). */
static const int EX[Q9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[Q9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

/* Side numbering for walls: 0 = -x, 1 = +x, 2 = -y, 3 = +y. Wall kinds. */
enum { ORC_PERIODIC = 0, ORC_DIRICHLET = 1, ORC_ADIABATIC = 2, ORC_WET = 3 };

typedef struct {
    int nx, ny;
    double nu, kappa, g_beta, T0, rho0;
    double s_b, s_3, s_4, lambda0, lambda2, cs2_T;
    double Fv[2];
    int wall[4];
    double T_wall[4];
    int thermal_only; /* 1: only the D2Q5 equation, with the velocity set by orc_set_velocity */
    double u_wall[4][2]; /* velocity of each wall (sides -x, +x, -y, +y) */
} orc_params;

typedef struct {
    orc_params p;
    double cs2;            /* lattice sound speed squared, 1/3 (Eq. 9) */
    double s_nu, lambda1;  /* from nu = (1/s_nu - 1/2) cs2 and alpha = (1/lambda1 - 1/2) cs2_T */
    double M[Q9][Q9], Minv[Q9][Q9], S[Q9][Q9];
    double MT[Q5][Q5], MTinv[Q5][Q5], ST[Q5][Q5];
    int opp[Q9];
    double wT[Q5];         /* D2Q5 rest weights, g^eq(T=1, u=0) */
    double fwall[4][Q9];   /* f^eq(rho0, u_wall) of each side */
    double gwall[4][Q5];   /* g^eq(T_wall, u_wall) of each side */
    double *f, *g;         /* pre-collision populations at the current time, [q][y][x] */
    double *fs, *gs;       /* post-collision scratch */
    double *uxp, *uyp;     /* prescribed velocity of the thermal-only mode, [y][x] */
    long steps;
} orc_sim;

/* ---------------------------------------------------------------- literal matrices (Eqs. 7, 17, 18) */

static void build_M(double M[Q9][Q9])
{
    /* Eq. (7a): rows k00, k10, k01, k20, k02, k11, k21, k12, k22 over populations 0..8. */
    static const double Mt[Q9][Q9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {0, 1, 0, -1, 0, 1, -1, -1, 1},
        {0, 0, 1, 0, -1, 1, 1, -1, -1},
        {0, 1, 0, 1, 0, 1, 1, 1, 1},
        {0, 0, 1, 0, 1, 1, 1, 1, 1},
        {0, 0, 0, 0, 0, 1, -1, 1, -1},
        {0, 0, 0, 0, 0, 1, 1, -1, -1},
        {0, 0, 0, 0, 0, 1, -1, -1, 1},
        {0, 0, 0, 0, 0, 1, 1, 1, 1},
    };
    memcpy(M, Mt, sizeof(Mt));
}

static void build_N(double ux, double uy, double N[Q9][Q9])
{
    /* Eq. (7b), with the k~02 row's k01 entry read as -2u_y (reading r1). */
    const double x = ux, y = uy, x2 = ux * ux, y2 = uy * uy;
    const double Nt[Q9][Q9] = {
        {1, 0, 0, 0, 0, 0, 0, 0, 0},
        {-x, 1, 0, 0, 0, 0, 0, 0, 0},
        {-y, 0, 1, 0, 0, 0, 0, 0, 0},
        {x2, -2 * x, 0, 1, 0, 0, 0, 0, 0},
        {y2, 0, -2 * y, 0, 1, 0, 0, 0, 0},
        {x * y, -y, -x, 0, 0, 1, 0, 0, 0},
        {-x2 * y, 2 * x * y, x2, -y, 0, -2 * x, 1, 0, 0},
        {-y2 * x, y2, 2 * x * y, 0, -x, -2 * y, 0, 1, 0},
        {x2 * y2, -2 * x * y2, -2 * y * x2, y2, x2, 4 * x * y, -2 * y, -2 * x, 1},
    };
    memcpy(N, Nt, sizeof(Nt));
}

static void build_MT(double M[Q5][Q5])
{
    /* Eq. (17): rows k00, k10, k01, k20, k02 over populations 0..4. */
    static const double Mt[Q5][Q5] = {
        {1, 1, 1, 1, 1},
        {0, 1, 0, -1, 0},
        {0, 0, 1, 0, -1},
        {0, 1, 0, 1, 0},
        {0, 0, 1, 0, 1},
    };
    memcpy(M, Mt, sizeof(Mt));
}

static void build_NT(double ux, double uy, double N[Q5][Q5])
{
    /* Eq. (18). */
    const double Nt[Q5][Q5] = {
        {1, 0, 0, 0, 0},
        {-ux, 1, 0, 0, 0},
        {-uy, 0, 1, 0, 0},
        {ux * ux, -2 * ux, 0, 1, 0},
        {uy * uy, 0, -2 * uy, 0, 1},
    };
    memcpy(N, Nt, sizeof(Nt));
}

/* ---------------------------------------------------------------- plain linear algebra */

/* Gauss-Jordan inverse with partial pivoting of an n x n row-major matrix. Returns 0 on success. */
static int invert(int n, const double *A, double *Ainv)
{
    double a[Q9 * 2 * Q9];
    const int w = 2 * n;
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < w; ++c)
            a[r * w + c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(a[r * w + c]) > fabs(a[piv * w + c])) piv = r;
        if (a[piv * w + c] == 0.0) return -1;
        if (piv != c)
            for (int k = 0; k < w; ++k) {
                double t = a[c * w + k];
                a[c * w + k] = a[piv * w + k];
                a[piv * w + k] = t;
            }
        const double d = a[c * w + c];
        for (int k = 0; k < w; ++k) a[c * w + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double m = a[r * w + c];
            for (int k = 0; k < w; ++k) a[r * w + k] -= m * a[c * w + k];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r * w + n + c];
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

/* Solve L x = b for unit lower-triangular L (this is how N^-1 and N_T^-1 are applied). */
static void solve_unit_lower(int n, const double *L, const double *b, double *x)
{
    for (int r = 0; r < n; ++r) {
        double s = b[r];
        for (int c = 0; c < r; ++c) s -= L[r * n + c] * x[c];
        x[r] = s;
    }
}

/* ---------------------------------------------------------------- set-up */

static void build_constants(orc_sim *s)
{
    const orc_params *p = &s->p;
    s->cs2 = 1.0 / 3.0;
    /* nu = (1/s_nu - 1/2) cs2 (Sec. 2.1) and alpha = (1/lambda1 - 1/2) cs2_T (Sec. 2.2). */
    s->s_nu = 1.0 / (p->nu / s->cs2 + 0.5);
    s->lambda1 = 1.0 / (p->kappa / p->cs2_T + 0.5);

    build_M(s->M);
    invert(Q9, &s->M[0][0], &s->Minv[0][0]);
    build_MT(s->MT);
    invert(Q5, &s->MT[0][0], &s->MTinv[0][0]);

    /* Relaxation matrix of Eq. (8): diag([0,0,0], [[s+,s-],[s-,s+]], [s_nu, s_3, s_3, s_4]). */
    memset(s->S, 0, sizeof(s->S));
    const double sp = 0.5 * (p->s_b + s->s_nu), sm = 0.5 * (p->s_b - s->s_nu);
    s->S[3][3] = sp; s->S[3][4] = sm;
    s->S[4][3] = sm; s->S[4][4] = sp;
    s->S[5][5] = s->s_nu;
    s->S[6][6] = p->s_3;
    s->S[7][7] = p->s_3;
    s->S[8][8] = p->s_4;
    /* D2Q5 relaxation matrix of Eq. (19): diag(lambda0, lambda1, lambda1, lambda2, lambda2). */
    memset(s->ST, 0, sizeof(s->ST));
    s->ST[0][0] = p->lambda0;
    s->ST[1][1] = s->lambda1;
    s->ST[2][2] = s->lambda1;
    s->ST[3][3] = p->lambda2;
    s->ST[4][4] = p->lambda2;

    /* Opposite directions found from the velocity set. */
    for (int i = 0; i < Q9; ++i)
        for (int j = 0; j < Q9; ++j)
            if (EX[j] == -EX[i] && EY[j] == -EY[i]) s->opp[i] = j;

    /* D2Q5 rest weights: g^eq = M_T^-1 N_T(0)^-1 [1, 0, 0, cs2_T, cs2_T] (Eqs. 20, 21). */
    const double geq[Q5] = {1.0, 0.0, 0.0, p->cs2_T, p->cs2_T};
    matvec(Q5, &s->MTinv[0][0], geq, s->wT);
}

/* ---------------------------------------------------------------- one node */

/* Macroscopic quantities of Eqs. (3), (13), (23) from pre-collision populations. */
static void macroscopic(const orc_sim *s, const double f[Q9], const double g[Q5], double *rho,
                        double *ux, double *uy, double *T, double *Fx, double *Fy)
{
    const orc_params *p = &s->p;
    double r = 0.0, jx = 0.0, jy = 0.0, t = 0.0;
    for (int i = 0; i < Q9; ++i) {
        r += f[i];
        jx += f[i] * EX[i];
        jy += f[i] * EY[i];
    }
    for (int i = 0; i < Q5; ++i) t += g[i];
    *Fx = p->Fv[0];
    *Fy = p->Fv[1] + p->rho0 * p->g_beta * (t - p->T0);
    *rho = r;
    *T = t;
    *ux = (jx + 0.5 * *Fx) / r;
    *uy = (jy + 0.5 * *Fy) / r;
}

/* Collision of one node: Eqs. (6)-(11) for f and Eqs. (16)-(21) for g. */
static void collide(const orc_sim *s, const double f[Q9], const double g[Q5], double fo[Q9],
                    double go[Q5])
{
    const orc_params *p = &s->p;
    double rho, ux, uy, T, Fx, Fy;
    macroscopic(s, f, g, &rho, &ux, &uy, &T, &Fx, &Fy);

    /* ---- D2Q9 ---- */
    double N[Q9][Q9];
    build_N(ux, uy, N);
    double gam[Q9], gt[Q9];
    matvec(Q9, &s->M[0][0], f, gam);     /* Gamma = M f            (Eq. 7a) */
    matvec(Q9, &N[0][0], gam, gt);       /* Gamma~ = N Gamma       (Eq. 7b) */
    const double cs2 = s->cs2;
    const double geq[Q9] = {rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2}; /* Eq. 9 */
    const double C[Q9] = {0, Fx, Fy, 0, 0, 0, cs2 * Fy, cs2 * Fx, 0};                  /* Eq. 11 */
    double d[Q9], Sd[Q9], SC[Q9], gts[Q9];
    for (int k = 0; k < Q9; ++k) d[k] = gt[k] - geq[k];
    matvec(Q9, &s->S[0][0], d, Sd);
    matvec(Q9, &s->S[0][0], C, SC);
    /* Eq. (8): Gamma~* = (I - S) Gamma~ + S Gamma~eq + (I - S/2) C */
    for (int k = 0; k < Q9; ++k) gts[k] = gt[k] - Sd[k] + C[k] - 0.5 * SC[k];
    double gams[Q9];
    solve_unit_lower(Q9, &N[0][0], gts, gams); /* Gamma* = N^-1 Gamma~* */
    matvec(Q9, &s->Minv[0][0], gams, fo);      /* f* = M^-1 Gamma*      */

    /* ---- D2Q5 ---- */
    double NT[Q5][Q5];
    build_NT(ux, uy, NT);
    double gamT[Q5], gtT[Q5];
    matvec(Q5, &s->MT[0][0], g, gamT);  /* Eq. 16 */
    matvec(Q5, &NT[0][0], gamT, gtT);
    const double c2 = p->cs2_T;
    const double geqT[Q5] = {T, 0, 0, T * c2, T * c2}; /* Eq. 20 */
    double dT[Q5], SdT[Q5], gtsT[Q5], gamsT[Q5];
    for (int k = 0; k < Q5; ++k) dT[k] = gtT[k] - geqT[k];
    matvec(Q5, &s->ST[0][0], dT, SdT);
    for (int k = 0; k < Q5; ++k) gtsT[k] = gtT[k] - SdT[k]; /* Eq. 19 */
    solve_unit_lower(Q5, &NT[0][0], gtsT, gamsT);
    matvec(Q5, &s->MTinv[0][0], gamsT, go);                 /* Eq. 21 */
}

/* D2Q5 collision alone, Eqs. (16)-(21), with a prescribed velocity (Sec. 3.1: the velocity field is
 * given and only the D2Q5 equation is solved). */
static void collide_thermal(const orc_sim *s, const double g[Q5], double ux, double uy, double go[Q5])
{
    const orc_params *p = &s->p;
    double T = 0.0;
    for (int i = 0; i < Q5; ++i) T += g[i];
    double NT[Q5][Q5];
    build_NT(ux, uy, NT);
    double gamT[Q5], gtT[Q5];
    matvec(Q5, &s->MT[0][0], g, gamT);
    matvec(Q5, &NT[0][0], gamT, gtT);
    const double c2 = p->cs2_T;
    const double geqT[Q5] = {T, 0, 0, T * c2, T * c2};
    double dT[Q5], SdT[Q5], gtsT[Q5], gamsT[Q5];
    for (int k = 0; k < Q5; ++k) dT[k] = gtT[k] - geqT[k];
    matvec(Q5, &s->ST[0][0], dT, SdT);
    for (int k = 0; k < Q5; ++k) gtsT[k] = gtT[k] - SdT[k];
    solve_unit_lower(Q5, &NT[0][0], gtsT, gamsT);
    matvec(Q5, &s->MTinv[0][0], gamsT, go);
}

/* Discrete equilibria: f^eq = M^-1 N(u)^-1 Gamma~eq(rho), g^eq = M_T^-1 N_T(u)^-1 Gamma~T,eq(T). */
static void equilibrium(const orc_sim *s, double rho, double ux, double uy, double T, double f[Q9],
                        double g[Q5])
{
    const double cs2 = s->cs2, c2 = s->p.cs2_T;
    double N[Q9][Q9], NT[Q5][Q5], gam[Q9], gamT[Q5];
    build_N(ux, uy, N);
    const double geq[Q9] = {rho, 0, 0, rho * cs2, rho * cs2, 0, 0, 0, rho * cs2 * cs2};
    solve_unit_lower(Q9, &N[0][0], geq, gam);
    matvec(Q9, &s->Minv[0][0], gam, f);
    build_NT(ux, uy, NT);
    const double geqT[Q5] = {T, 0, 0, T * c2, T * c2};
    solve_unit_lower(Q5, &NT[0][0], geqT, gamT);
    matvec(Q5, &s->MTinv[0][0], gamT, g);
}

/* ---------------------------------------------------------------- lattice */

static size_t nodes(const orc_sim *s) { return (size_t)s->p.nx * (size_t)s->p.ny; }

/* Streaming, Eqs. (12) and (22), pulled: population i at x comes from x - e_i. When x - e_i lies
 * beyond a wall, the boundary rule of reading r10 supplies it from the node's own post-collision
 * populations. Periodic sides wrap. */
static void equilibrium(const orc_sim *s, double rho, double ux, double uy, double T, double f[Q9],
                        double g[Q5]);

/* Equilibria of the walls, used by the moving-wall bounce-back and the anti-bounce-back:
 * f_i = f*_opp + [f^eq_i - f^eq_opp](rho0, u_w) and g_i = -g*_opp + [g^eq_i + g^eq_opp](T_w, u_w)
 * (reading r10; at u_w = 0 they reduce to plain bounce-back and g_i = -g*_opp + 2 w^T_i T_w). */
static void wall_equilibria(orc_sim *s)
{
    for (int side = 0; side < 4; ++side)
        equilibrium(s, s->p.rho0, s->p.u_wall[side][0], s->p.u_wall[side][1], s->p.T_wall[side],
                    s->fwall[side], s->gwall[side]);
}

static void stream(orc_sim *s)
{
    const orc_params *p = &s->p;
    const int nx = p->nx, ny = p->ny;
    const size_t n = nodes(s);
#pragma omp parallel for schedule(static) if (n >= ORC_OMP_MIN_NODES)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            const size_t here = (size_t)y * nx + x;
            for (int i = 0; i < Q9; ++i) {
                int sx = x - EX[i], sy = y - EY[i];
                int side = -1; /* wall crossed, if any; for a corner the y wall is recorded last */
                if (sx < 0) { if (p->wall[0] == ORC_PERIODIC) sx += nx; else side = 0; }
                if (sx >= nx) { if (p->wall[1] == ORC_PERIODIC) sx -= nx; else side = 1; }
                if (sy < 0) { if (p->wall[2] == ORC_PERIODIC) sy += ny; else side = 2; }
                if (sy >= ny) { if (p->wall[3] == ORC_PERIODIC) sy -= ny; else side = 3; }
                const int o = s->opp[i];
                if (side < 0) {
                    const size_t src = (size_t)sy * nx + sx;
                    s->f[i * n + here] = s->fs[i * n + src];
                    if (i < Q5) s->g[i * n + here] = s->gs[i * n + src];
                } else {
                    /* halfway bounce-back, with the wall's momentum when it moves */
                    s->f[i * n + here] = s->fs[o * n + here] + (s->fwall[side][i] - s->fwall[side][o]);
                    if (i < Q5) {
                        if (p->wall[side] == ORC_DIRICHLET) /* anti-bounce-back */
                            s->g[i * n + here] = -s->gs[o * n + here] + (s->gwall[side][i] + s->gwall[side][o]);
                        else                                /* adiabatic: bounce-back */
                            s->g[i * n + here] = s->gs[o * n + here];
                    }
                }
            }
        }
}

/* One node on a wet wall (reading r19 on y sides, r26 on x sides and in corners), on the streamed
 * (pre-collision) state: non-equilibrium bounce-back for f, non-equilibrium extrapolation for g from
 * the fluid node q next to it (along the wall's normal; at a corner, the diagonal neighbour). Reads
 * only the node's own streamed values and q's, and q is never a wall node (nx, ny >= 3), so the
 * wall nodes can be processed in any order. */
static void wet_node(orc_sim *s, int x, int y, int onx, int ony)
{
    const orc_params *p = &s->p;
    const int nx = p->nx;
    const size_t n = nodes(s);
    const int sx = x == 0 ? 1 : -1, sy = y == 0 ? 1 : -1; /* directions into the fluid */
    const int side_x = x == 0 ? 0 : 1, side_y = y == 0 ? 2 : 3;
    const int side = ony ? side_y : side_x;
    /* a corner takes the y wall's velocity and the mean of the two walls' temperatures */
    const double uwx = p->u_wall[side][0], uwy = p->u_wall[side][1];
    const double Tw = (onx && ony) ? 0.5 * (p->T_wall[side_x] + p->T_wall[side_y]) : p->T_wall[side];
    const int qx = onx ? x + sx : x, qy = ony ? y + sy : y;
    const size_t b = (size_t)y * nx + x, q = (size_t)qy * nx + qx;
    double f[Q9], g[Q5], fq[Q9], gq[Q5];
    for (int i = 0; i < Q9; ++i) f[i] = s->f[i * n + b];
    for (int i = 0; i < Q9; ++i) fq[i] = s->f[i * n + q];
    for (int i = 0; i < Q5; ++i) gq[i] = s->g[i * n + q];
    double rq, uqx, uqy, Tq, Fqx, Fqy;
    macroscopic(s, fq, gq, &rq, &uqx, &uqy, &Tq, &Fqx, &Fqy);
    if (p->thermal_only) {
        uqx = s->uxp[q];
        uqy = s->uyp[q];
    } else {
        const double Fx = p->Fv[0], Fy = p->Fv[1] + p->rho0 * p->g_beta * (Tw - p->T0);
        double rho, feq[Q9], gdum[Q5];
        if (onx && ony) {
            /* corner: rho from the diagonal neighbour; the unknowns whose opposite is known by
             * non-equilibrium bounce-back; the two buried diagonals share the remaining mass */
            rho = rq;
            equilibrium(s, rho, uwx - 0.5 * Fx / rho, uwy - 0.5 * Fy / rho, Tw, feq, gdum);
            int unknown[Q9];
            for (int i = 0; i < Q9; ++i) unknown[i] = EX[i] == sx || EY[i] == sy;
            double known = 0.0;
            for (int i = 0; i < Q9; ++i) {
                const int o = s->opp[i];
                if (unknown[i] && !unknown[o]) f[i] = f[o] + (feq[i] - feq[o]);
                if (!(unknown[i] && unknown[o])) known += f[i];
            }
            for (int i = 0; i < Q9; ++i)
                if (unknown[i] && unknown[s->opp[i]]) f[i] = 0.5 * (rho - known);
        } else {
            /* one wall with normal along axis a: rho from mass and normal momentum, the unknowns
             * by non-equilibrium bounce-back, the tangential momentum closed on the two diagonals */
            const int *Ea = onx ? EX : EY, *Et = onx ? EY : EX;
            const int nrm = onx ? sx : sy;
            const double Fa = onx ? Fx : Fy, uwa = onx ? uwx : uwy;
            double Z = 0.0, O = 0.0;
            for (int i = 0; i < Q9; ++i) {
                if (Ea[i] == 0) Z += f[i];
                if (Ea[i] == -nrm) O += f[i];
            }
            rho = (Z + 2.0 * O - nrm * 0.5 * Fa) / (1.0 - nrm * uwa);
            const double upx = uwx - 0.5 * Fx / rho, upy = uwy - 0.5 * Fy / rho;
            equilibrium(s, rho, upx, upy, Tw, feq, gdum);
            for (int i = 0; i < Q9; ++i)
                if (Ea[i] == nrm) f[i] = f[s->opp[i]] + (feq[i] - feq[s->opp[i]]);
            double St = 0.0;
            for (int i = 0; i < Q9; ++i) St += f[i] * Et[i];
            const double delta = 0.5 * (rho * (onx ? upy : upx) - St);
            for (int i = 0; i < Q9; ++i)
                if (Ea[i] == nrm && Et[i] != 0) f[i] += Et[i] * delta;
        }
        for (int i = 0; i < Q9; ++i) s->f[i * n + b] = f[i];
    }
    /* temperature: g_i = g^eq_i(T_w, u_w) + [g_i(q) - g^eq_i(T(q), u(q))]; in the thermal-only
     * mode u is the prescribed velocity of the node and of q */
    const double ubx = p->thermal_only ? s->uxp[b] : uwx, uby = p->thermal_only ? s->uyp[b] : uwy;
    double fe[Q9], geqq[Q5], geqb[Q5];
    equilibrium(s, rq, uqx, uqy, Tq, fe, geqq);
    equilibrium(s, 1.0, ubx, uby, Tw, fe, geqb);
    for (int i = 0; i < Q5; ++i) g[i] = geqb[i] + (gq[i] - geqq[i]);
    for (int i = 0; i < Q5; ++i) s->g[i * n + b] = g[i];
}

/* The wet-wall boundary pass on the streamed (pre-collision) state. */
static void apply_wet_walls(orc_sim *s)
{
    const orc_params *p = &s->p;
    const int wx = p->wall[0] == ORC_WET, wy = p->wall[2] == ORC_WET;
    if (!wx && !wy) return;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            const int onx = wx && (x == 0 || x == p->nx - 1), ony = wy && (y == 0 || y == p->ny - 1);
            if (onx || ony) wet_node(s, x, y, onx, ony);
        }
}

static void collide_all(orc_sim *s)
{
    const long n = (long)nodes(s);
#pragma omp parallel for schedule(static) if (n >= ORC_OMP_MIN_NODES)
    for (long k = 0; k < n; ++k) {
        double f[Q9], g[Q5], fo[Q9], go[Q5];
        for (int i = 0; i < Q9; ++i) f[i] = s->f[i * n + k];
        for (int i = 0; i < Q5; ++i) g[i] = s->g[i * n + k];
        if (s->p.thermal_only) {
            for (int i = 0; i < Q9; ++i) fo[i] = f[i];
            collide_thermal(s, g, s->uxp[k], s->uyp[k], go);
        } else {
            collide(s, f, g, fo, go);
        }
        for (int i = 0; i < Q9; ++i) s->fs[i * n + k] = fo[i];
        for (int i = 0; i < Q5; ++i) s->gs[i * n + k] = go[i];
    }
}

/* ---------------------------------------------------------------- exported API (ctypes) */

int orc_create(const orc_params *p, orc_sim **out)
{
    *out = NULL;
    if (p->nx < 2 || p->ny < 2) return -1;
    /* wet walls come in pairs (both x sides, or both y sides), need three nodes across, and the
     * other pair of sides is periodic or wet as well */
    for (int a = 0; a < 2; ++a) {
        const int lo = p->wall[2 * a], hi = p->wall[2 * a + 1], other = p->wall[2 - 2 * a];
        if ((lo == ORC_WET) != (hi == ORC_WET)) return -1;
        if (lo == ORC_WET && ((a == 0 ? p->nx : p->ny) < 3 || (other != ORC_PERIODIC && other != ORC_WET)))
            return -1;
    }
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return -2;
    s->p = *p;
    build_constants(s);
    wall_equilibria(s);
    const size_t n = nodes(s);
    s->f = (double *)calloc(Q9 * n, sizeof(double));
    s->fs = (double *)calloc(Q9 * n, sizeof(double));
    s->g = (double *)calloc(Q5 * n, sizeof(double));
    s->gs = (double *)calloc(Q5 * n, sizeof(double));
    s->uxp = (double *)calloc(n, sizeof(double));
    s->uyp = (double *)calloc(n, sizeof(double));
    if (!s->f || !s->fs || !s->g || !s->gs || !s->uxp || !s->uyp) {
        free(s->f); free(s->fs); free(s->g); free(s->gs); free(s->uxp); free(s->uyp); free(s);
        return -2;
    }
    *out = s;
    return 0;
}

void orc_destroy(orc_sim *s)
{
    if (!s) return;
    free(s->f); free(s->fs); free(s->g); free(s->gs); free(s->uxp); free(s->uyp);
    free(s);
}

/* f(x,0) = f^eq(rho, u), g(x,0) = g^eq(T, u) from row-major [ny][nx] fields. */
void orc_init(orc_sim *s, const double *rho, const double *ux, const double *uy, const double *T)
{
    const size_t n = nodes(s);
    if (s->p.thermal_only) {
        memcpy(s->uxp, ux, n * sizeof(double));
        memcpy(s->uyp, uy, n * sizeof(double));
    }
    for (size_t k = 0; k < n; ++k) {
        double f[Q9], g[Q5];
        equilibrium(s, rho[k], ux[k], uy[k], T[k], f, g);
        for (int i = 0; i < Q9; ++i) s->f[i * n + k] = f[i];
        for (int i = 0; i < Q5; ++i) s->g[i * n + k] = g[i];
    }
    apply_wet_walls(s);
    s->steps = 0;
}

void orc_step(orc_sim *s, long nsteps)
{
    for (long t = 0; t < nsteps; ++t) {
        collide_all(s);
        stream(s);
        apply_wet_walls(s);
        s->steps++;
    }
}

long orc_steps(const orc_sim *s) { return s->steps; }

/* Threads the node loops run on (1 without OpenMP). The arithmetic per node does not depend on it. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_fields(const orc_sim *s, double *rho, double *ux, double *uy, double *T)
{
    const size_t n = nodes(s);
    for (size_t k = 0; k < n; ++k) {
        double f[Q9], g[Q5], Fx, Fy;
        for (int i = 0; i < Q9; ++i) f[i] = s->f[i * n + k];
        for (int i = 0; i < Q5; ++i) g[i] = s->g[i * n + k];
        macroscopic(s, f, g, &rho[k], &ux[k], &uy[k], &T[k], &Fx, &Fy);
        if (s->p.thermal_only) {
            ux[k] = s->uxp[k];
            uy[k] = s->uyp[k];
        }
    }
}

void orc_get_pops(const orc_sim *s, double *f, double *g)
{
    const size_t n = nodes(s);
    memcpy(f, s->f, Q9 * n * sizeof(double));
    memcpy(g, s->g, Q5 * n * sizeof(double));
}

void orc_set_pops(orc_sim *s, const double *f, const double *g)
{
    const size_t n = nodes(s);
    memcpy(s->f, f, Q9 * n * sizeof(double));
    memcpy(s->g, g, Q5 * n * sizeof(double));
}

/* Per-node primitives, used by the pins. */
int orc_collide_node(const orc_params *p, const double *f, const double *g, double *fo, double *go)
{
    orc_sim s;
    memset(&s, 0, sizeof(s));
    s.p = *p;
    build_constants(&s);
    collide(&s, f, g, fo, go);
    return 0;
}

int orc_equilibrium_node(const orc_params *p, double rho, double ux, double uy, double T,
                         double *f, double *g)
{
    orc_sim s;
    memset(&s, 0, sizeof(s));
    s.p = *p;
    build_constants(&s);
    equilibrium(&s, rho, ux, uy, T, f, g);
    return 0;
}

int orc_collide_thermal_node(const orc_params *p, const double *g, double ux, double uy, double *go)
{
    orc_sim s;
    memset(&s, 0, sizeof(s));
    s.p = *p;
    build_constants(&s);
    collide_thermal(&s, g, ux, uy, go);
    return 0;
}

/* The matrices as the oracle uses them: M, M^-1, N(u), N(u)^-1 (by solving against unit vectors),
 * M_T, M_T^-1, N_T(u), N_T(u)^-1, the relaxation matrices S, S_T and the D2Q5 rest weights. */
void orc_matrices(const orc_params *p, double ux, double uy, double *M, double *Minv, double *N,
                  double *Ninv, double *MT, double *MTinv, double *NT, double *NTinv, double *S,
                  double *ST, double *wT)
{
    orc_sim s;
    memset(&s, 0, sizeof(s));
    s.p = *p;
    build_constants(&s);
    double Nl[Q9][Q9], NTl[Q5][Q5];
    build_N(ux, uy, Nl);
    build_NT(ux, uy, NTl);
    memcpy(M, s.M, sizeof(s.M));
    memcpy(Minv, s.Minv, sizeof(s.Minv));
    memcpy(N, Nl, sizeof(Nl));
    memcpy(MT, s.MT, sizeof(s.MT));
    memcpy(MTinv, s.MTinv, sizeof(s.MTinv));
    memcpy(NT, NTl, sizeof(NTl));
    memcpy(S, s.S, sizeof(s.S));
    memcpy(ST, s.ST, sizeof(s.ST));
    memcpy(wT, s.wT, sizeof(s.wT));
    for (int c = 0; c < Q9; ++c) {
        double e[Q9] = {0}, col[Q9];
        e[c] = 1.0;
        solve_unit_lower(Q9, &Nl[0][0], e, col);
        for (int r = 0; r < Q9; ++r) Ninv[r * Q9 + c] = col[r];
    }
    for (int c = 0; c < Q5; ++c) {
        double e[Q5] = {0}, col[Q5];
        e[c] = 1.0;
        solve_unit_lower(Q5, &NTl[0][0], e, col);
        for (int r = 0; r < Q5; ++r) NTinv[r * Q5 + c] = col[r];
    }
}
