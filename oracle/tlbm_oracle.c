/*
 * tlbm_oracle.c -- plain, slow, FP64 CPU oracle of one time step of the ternary
 * free-energy lattice Boltzmann method of Semprebon, Krueger and Kusumaatmaja,
 * "Ternary free energy lattice Boltzmann model with tunable surface tensions and
 * contact angles" (arXiv:1511.02155).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this file.  The GPU product path never
 * calls it, and it shares no code, header, table or helper with the GPU path.
 *
 * Every quantity is IEEE double.  The file is compiled with -ffp-contract=off so
 * that no multiply-add is fused.  Every sum runs in ascending index order.
 *
 * One step, in the paper's order (Sec. "The Lattice Boltzmann Equation"):
 *   O1 moments           rho = sum f, rho v = sum f e, phi = sum g, psi = sum k
 *                        (Eq. lbconstraint)
 *   O2 wetting ghosts    solid nodes next to fluid get values that impose the
 *                        Neumann conditions of the wetting section
 *                        (Sec. Auxiliary variables, gradients of rho/phi/psi)
 *   O3 derivatives       isotropic lattice-weight gradient and Laplacian
 *   O4 thermodynamics    C_m, mu_m, mu_rho, mu_phi, mu_psi, p_b
 *                        (Sec. Auxiliary variables; Sec. Equations of Motion)
 *   O5 equilibria        f_eq, g_eq, k_eq for i > 0 (Eq. eqdistfbinary and the
 *                        g/k equilibria beneath it), rest populations from the
 *                        mass constraints that close the LBM section
 *   O6 BGK collision     Eq. latboltCollision
 *   O7 streaming         Eq. latboltPropagation, pull form, halfway bounce-back
 *                        at solid nodes ("standard bounce back")
 *   O8 mass totals       Kahan-summed sums of rho, phi, psi over fluid nodes
 *
 * The forcing coupling (orc_step_guo), the alternative that Sec. Equations of
 * Motion mentions beside the pressure-tensor route (Guo forcing): the
 * thermodynamic terms enter the momentum equation as a body force.  In the
 * continuum it is F = -(rho grad mu_rho + phi grad mu_phi + psi grad mu_psi),
 * the last three
 * terms of the Navier-Stokes equation, which the paper writes as the divergence
 * of its pressure tensor minus the ideal-gas pressure; on the lattice it is
 * taken in that divergence form,
 *   F_a = -d_b (P_ab - rho c_s^2 delta_ab),
 * P_ab node by node from O3-O4 (the printed pressure tensor, with p_b, alpha^2
 * and the symmetric cross terms read as listed below)
 * and d_b by the isotropic gradient stencil of O3, so that the total momentum
 * is conserved exactly on a periodic lattice.  f relaxes to the ideal-gas
 * equilibrium (pressure rho c_s^2) at u = (rho v + F/2) / rho and receives the
 * source of Guo, Zheng and Shi (2002):
 *   (1 - 1/(2 tau)) w_i [(e_i - u).F / c_s^2 + (e_i.u)(e_i.F) / c_s^4];
 * g and k keep their equilibria, evaluated at the same u.  Periodic lattices.
 *
 * Readings taken where the paper is silent or misprinted (each pinned by a test):
 *   - mu_rho is the functional derivative dF/drho, i.e. (mu_1 + mu_2)/2; the
 *     printed mu_rho has a sign and a Laplacian mix-up.  mu_phi and mu_psi match
 *     the printed forms.
 *   - p_b is the thermodynamic identity sum_X X df_b/dX - f_b + rho c_s^2, i.e.
 *     rho/3 + sum_m kappa_m/2 C_m^2 (1-C_m)(1-3C_m); the printed polynomial has an
 *     extra 3 kappa_3 psi^2 / 2.
 *   - the gradient terms of f_eq carry the alpha^2 of the pressure tensor, and the
 *     duplicated cross terms are read in their symmetric form.
 *   - D3Q19 index order follows the weight table; D2Q9 tensors are the standard
 *     binary free-energy set scaled to the same normalisation as the D3Q19 table.
 *   - derivative stencils: d_a X = (1/c_s^2) sum_i w_i e_ia X(r+e_i),
 *     lap X = (2/c_s^2) sum_i w_i (X(r+e_i) - X(r)).
 *   - Gamma_phi, Gamma_psi are parameters; tau_X = 1/2 + M_X / Gamma_X is set by
 *     the caller.
 *   - wetting ghost rule: a solid node with fluid axis-neighbours takes the mean of
 *     X(n) - G_X over them; with only diagonal fluid neighbours, the mean of
 *     X(n) - sqrt(2) G_X; G_X is the wall-normal gradient of the wetting section.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int Q;              /* 9 (D2Q9) or 19 (D3Q19) */
    int nx, ny, nz;     /* lattice size; nz = 1 for D2Q9 */
    double kappa[3];    /* kappa_1..3 */
    double alpha;       /* interface width */
    double tau[3];      /* tau_rho (tau_f), tau_phi, tau_psi */
    double gamma[2];    /* Gamma_phi, Gamma_psi */
    double h[3];        /* wetting parameters h_1..3 */
} orc_params;

/* ---------------------------------------------------------------- lattices */

/* D2Q9: rest, four axis directions, four diagonals. */
static const int E9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {-1, 1, 0}, {1, -1, 0}};
static const double W9[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
/* gradient-term tensors w_i^{ab}, components ordered xx yy zz xy yz zx */
static const double T9[9][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 9.0, -1.0 / 18.0, 0, 0, 0, 0},
    {1.0 / 9.0, -1.0 / 18.0, 0, 0, 0, 0},
    {-1.0 / 18.0, 1.0 / 9.0, 0, 0, 0, 0},
    {-1.0 / 18.0, 1.0 / 9.0, 0, 0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 0, 1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 0, 1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 0, -1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 0, -1.0 / 12.0, 0, 0}};

/* D3Q19 in the order implied by the paper's weight table. */
static const int E19[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},  {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {1, -1, 0}, {-1, 1, 0}, {-1, -1, 0}, {0, 1, 1},   {0, 1, -1}, {0, -1, 1},
    {0, -1, -1}, {1, 0, 1}, {1, 0, -1}, {-1, 0, 1},  {-1, 0, -1}};
static const double W19[19] = {
    1.0 / 3.0,  1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double T19[19][6] = {
    {0, 0, 0, 0, 0, 0},
    /* 1,2: +-x */
    {5.0 / 36.0, -1.0 / 9.0, -1.0 / 9.0, 0, 0, 0},
    {5.0 / 36.0, -1.0 / 9.0, -1.0 / 9.0, 0, 0, 0},
    /* 3,4: +-y */
    {-1.0 / 9.0, 5.0 / 36.0, -1.0 / 9.0, 0, 0, 0},
    {-1.0 / 9.0, 5.0 / 36.0, -1.0 / 9.0, 0, 0, 0},
    /* 5,6: +-z */
    {-1.0 / 9.0, -1.0 / 9.0, 5.0 / 36.0, 0, 0, 0},
    {-1.0 / 9.0, -1.0 / 9.0, 5.0 / 36.0, 0, 0, 0},
    /* 7..10: xy edges */
    {-1.0 / 72.0, -1.0 / 72.0, 1.0 / 36.0, 1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 1.0 / 36.0, -1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 1.0 / 36.0, -1.0 / 12.0, 0, 0},
    {-1.0 / 72.0, -1.0 / 72.0, 1.0 / 36.0, 1.0 / 12.0, 0, 0},
    /* 11..14: yz edges */
    {1.0 / 36.0, -1.0 / 72.0, -1.0 / 72.0, 0, 1.0 / 12.0, 0},
    {1.0 / 36.0, -1.0 / 72.0, -1.0 / 72.0, 0, -1.0 / 12.0, 0},
    {1.0 / 36.0, -1.0 / 72.0, -1.0 / 72.0, 0, -1.0 / 12.0, 0},
    {1.0 / 36.0, -1.0 / 72.0, -1.0 / 72.0, 0, 1.0 / 12.0, 0},
    /* 15..18: zx edges */
    {-1.0 / 72.0, 1.0 / 36.0, -1.0 / 72.0, 0, 0, 1.0 / 12.0},
    {-1.0 / 72.0, 1.0 / 36.0, -1.0 / 72.0, 0, 0, -1.0 / 12.0},
    {-1.0 / 72.0, 1.0 / 36.0, -1.0 / 72.0, 0, 0, -1.0 / 12.0},
    {-1.0 / 72.0, 1.0 / 36.0, -1.0 / 72.0, 0, 0, 1.0 / 12.0}};

typedef struct {
    int Q, D;                 /* velocities, dimension */
    int naxis;                /* number of axis directions (2D) */
    const int (*e)[3];
    const double *w;
    const double (*t)[6];
    int opp[19];
    int nx, ny, nz;
    size_t N;
} lattice;

static int lattice_init(lattice *L, const orc_params *p)
{
    if (p->Q == 9) {
        L->Q = 9; L->D = 2; L->e = E9; L->w = W9; L->t = T9;
        if (p->nz != 1) return -1;
    } else if (p->Q == 19) {
        L->Q = 19; L->D = 3; L->e = E19; L->w = W19; L->t = T19;
    } else {
        return -1;
    }
    L->naxis = 2 * L->D;
    for (int i = 0; i < L->Q; ++i) {
        L->opp[i] = -1;
        for (int j = 0; j < L->Q; ++j)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1] && L->e[j][2] == -L->e[i][2])
                L->opp[i] = j;
    }
    L->nx = p->nx; L->ny = p->ny; L->nz = p->nz;
    if (L->nx < 1 || L->ny < 1 || L->nz < 1) return -1;
    L->N = (size_t)L->nx * (size_t)L->ny * (size_t)L->nz;
    return 0;
}

/* node index of r + s*e_i with periodic wrap; s = +1 or -1 */
static size_t shift(const lattice *L, size_t r, int i, int s)
{
    long x = (long)(r % (size_t)L->nx);
    long y = (long)((r / (size_t)L->nx) % (size_t)L->ny);
    long z = (long)(r / ((size_t)L->nx * (size_t)L->ny));
    x = (x + s * L->e[i][0]) % L->nx; if (x < 0) x += L->nx;
    y = (y + s * L->e[i][1]) % L->ny; if (y < 0) y += L->ny;
    z = (z + s * L->e[i][2]) % L->nz; if (z < 0) z += L->nz;
    return (size_t)x + (size_t)L->nx * ((size_t)y + (size_t)L->ny * (size_t)z);
}

static int is_solid(const uint8_t *solid, size_t r) { return solid != NULL && solid[r] != 0; }

/* exported lattice tables (for the tensor-identity tests) */
int orc_lattice(int Q, int *e, double *w, double *t, int *opp)
{
    orc_params p; memset(&p, 0, sizeof p);
    p.Q = Q; p.nx = p.ny = p.nz = 1;
    lattice L;
    if (lattice_init(&L, &p) != 0) return -1;
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = L.e[i][a];
        w[i] = L.w[i];
        for (int c = 0; c < 6; ++c) t[6 * i + c] = L.t[i][c];
        opp[i] = L.opp[i];
    }
    return 0;
}

/* ------------------------------------------------------- O4 thermodynamics */

/* mixing coefficients kappa_XY of the pressure tensor, X,Y in {rho,phi,psi} */
static void mixing(const orc_params *p, double K[3][3])
{
    const double k1 = p->kappa[0], k2 = p->kappa[1], k3 = p->kappa[2];
    K[0][0] = (k1 + k2) / 4.0;             /* rho rho */
    K[1][1] = (k1 + k2) / 4.0;             /* phi phi */
    K[2][2] = (k1 + k2 + 4.0 * k3) / 4.0;  /* psi psi */
    K[0][1] = K[1][0] = (k1 - k2) / 4.0;   /* rho phi */
    K[1][2] = K[2][1] = -(k1 - k2) / 4.0;  /* phi psi */
    K[0][2] = K[2][0] = -(k1 + k2) / 4.0;  /* rho psi */
}

/*
 * Local thermodynamics at one node (Sec. Auxiliary variables; Sec. Equations of
 * Motion).  X = (rho, phi, psi), lap = Laplacians of X.
 * Out: C[3] = C_1..3, mu[3] = (mu_rho, mu_phi, mu_psi), *pb = bulk pressure.
 */
void orc_thermo_node(const orc_params *p, const double X[3], const double lap[3],
                     double C[3], double mu[3], double *pb)
{
    const double a2 = p->alpha * p->alpha;
    double lapC[3], muC[3];
    C[0] = (X[0] + X[1] - X[2]) / 2.0;
    C[1] = (X[0] - X[1] - X[2]) / 2.0;
    C[2] = X[2];
    lapC[0] = (lap[0] + lap[1] - lap[2]) / 2.0;
    lapC[1] = (lap[0] - lap[1] - lap[2]) / 2.0;
    lapC[2] = lap[2];
    for (int m = 0; m < 3; ++m) {
        const double c = C[m];
        muC[m] = p->kappa[m] * c * (1.0 - c) * (1.0 - 2.0 * c) - a2 * p->kappa[m] * lapC[m];
    }
    mu[0] = (muC[0] + muC[1]) / 2.0;
    mu[1] = (muC[0] - muC[1]) / 2.0;
    mu[2] = muC[2] - (muC[0] + muC[1]) / 2.0;
    double s = X[0] / 3.0;
    for (int m = 0; m < 3; ++m) {
        const double c = C[m];
        s += p->kappa[m] / 2.0 * c * c * (1.0 - c) * (1.0 - 3.0 * c);
    }
    *pb = s;
}

/* -------------------------------------------------------- O5 equilibria */

/*
 * Equilibria at one fluid node (Eq. eqdistfbinary and the g, k equilibria).
 * X = (rho, phi, psi); j = rho v; grad[f][a] = d_a of field f; lap[f].
 * Directions i >= 1 follow the printed forms; i = 0 closes sum_i x_eq = X.
 */
void orc_equilibrium_node(const orc_params *p, const double X[3], const double j[3],
                          const double grad[3][3], const double lap[3],
                          double *feq, double *geq, double *keq)
{
    lattice L;
    orc_params q = *p; q.nx = q.ny = q.nz = 1;
    lattice_init(&L, &q);
    const double cs2 = 1.0 / 3.0;
    const double a2 = p->alpha * p->alpha;
    double C[3], mu[3], pb;
    orc_thermo_node(p, X, lap, C, mu, &pb);
    double K[3][3];
    mixing(p, K);

    const double rho = X[0], phi = X[1], psi = X[2];
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];

    /* Laplacian part: sum_X K_XX X lap X + sum_{X<Y} K_XY (X lap Y + Y lap X) */
    double Lap = 0.0;
    for (int a = 0; a < 3; ++a) Lap += K[a][a] * X[a] * lap[a];
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b) Lap += K[a][b] * (X[a] * lap[b] + X[b] * lap[a]);

    /* gradient part G_ab, components xx yy zz xy yz zx */
    static const int ca[6] = {0, 1, 2, 0, 1, 2};
    static const int cb[6] = {0, 1, 2, 1, 2, 0};
    double G[6];
    for (int c = 0; c < 6; ++c) {
        const int al = ca[c], be = cb[c];
        double s = 0.0;
        for (int x = 0; x < 3; ++x) s += K[x][x] * grad[x][al] * grad[x][be];
        for (int x = 0; x < 3; ++x)
            for (int y = x + 1; y < 3; ++y)
                s += K[x][y] * (grad[x][al] * grad[y][be] + grad[x][be] * grad[y][al]);
        G[c] = s;
    }

    double sf = 0.0, sg = 0.0, sk = 0.0;
    for (int i = 1; i < L.Q; ++i) {
        double eu = 0.0;
        for (int a = 0; a < 3; ++a) eu += L.e[i][a] * u[a];
        const double quad = (eu * eu - cs2 * uu) / (2.0 * cs2 * cs2);
        double tg = 0.0;
        for (int c = 0; c < 6; ++c) tg += L.t[i][c] * G[c];
        const double wi = L.w[i];
        feq[i] = wi * (pb / cs2 + rho * eu / cs2 + rho * quad)
               - wi / cs2 * a2 * Lap
               + a2 / cs2 * tg;
        geq[i] = wi * (p->gamma[0] * mu[1] / cs2 + phi * eu / cs2 + phi * quad);
        keq[i] = wi * (p->gamma[1] * mu[2] / cs2 + psi * eu / cs2 + psi * quad);
        sf += feq[i]; sg += geq[i]; sk += keq[i];
    }
    feq[0] = rho - sf;
    geq[0] = phi - sg;
    keq[0] = psi - sk;
}

/* ------------------------------------------------------------ O1 moments */

/* Moments of conventional populations (Eq. lbconstraint) at fluid nodes; solid
 * nodes get zeros.  Any output pointer may be NULL except rho/phi/psi. */
void orc_moments(const orc_params *p, const uint8_t *solid, const double *f, const double *g,
                 const double *k, double *rho, double *jx, double *jy, double *jz,
                 double *phi, double *psi)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return;
    const size_t N = L.N;
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        double sr = 0, sx = 0, sy = 0, sz = 0, sp = 0, ss = 0;
        if (!is_solid(solid, r)) {
            for (int i = 0; i < L.Q; ++i) {
                const double fi = f[(size_t)i * N + r];
                sr += fi;
                sx += fi * L.e[i][0];
                sy += fi * L.e[i][1];
                sz += fi * L.e[i][2];
                sp += g[(size_t)i * N + r];
                ss += k[(size_t)i * N + r];
            }
        }
        rho[r] = sr; phi[r] = sp; psi[r] = ss;
        if (jx) jx[r] = sx;
        if (jy) jy[r] = sy;
        if (jz) jz[r] = sz;
    }
}

/* ------------------------------------------------------- O2 wetting ghosts */

/* wall-normal gradients of rho, phi, psi imposed by the wetting parameters */
void orc_wetting_gradients(const orc_params *p, double G[3])
{
    const double a2 = p->alpha * p->alpha;
    const double q1 = p->h[0] / (a2 * p->kappa[0]);
    const double q2 = p->h[1] / (a2 * p->kappa[1]);
    const double q3 = p->h[2] / (a2 * p->kappa[2]);
    G[0] = -q1 - q2 - q3;
    G[1] = -q1 + q2;
    G[2] = -q3;
}

/* Fill X = (rho, phi, psi) on solid nodes from fluid neighbours (rule in the
 * header); solid nodes with no fluid neighbour get 0. */
void orc_ghosts(const orc_params *p, const uint8_t *solid, double *rho, double *phi, double *psi)
{
    lattice L;
    if (lattice_init(&L, p) != 0 || solid == NULL) return;
    double G[3];
    orc_wetting_gradients(p, G);
    double *F[3] = {rho, phi, psi};
    const size_t N = L.N;
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t s = (size_t)rr;
        if (!solid[s]) continue;
        double acc[3] = {0, 0, 0};
        int n = 0;
        for (int i = 1; i <= L.naxis; ++i) {
            const size_t b = shift(&L, s, i, +1);
            if (solid[b]) continue;
            for (int c = 0; c < 3; ++c) acc[c] += F[c][b] - G[c];
            ++n;
        }
        if (n == 0) {
            const double r2 = sqrt(2.0);
            for (int i = L.naxis + 1; i < L.Q; ++i) {
                const size_t b = shift(&L, s, i, +1);
                if (solid[b]) continue;
                for (int c = 0; c < 3; ++c) acc[c] += F[c][b] - r2 * G[c];
                ++n;
            }
        }
        for (int c = 0; c < 3; ++c) F[c][s] = n > 0 ? acc[c] / (double)n : 0.0;
    }
}

/* ------------------------------------------------------- O3 derivatives */

/* gradient and Laplacian of one field at node r (neighbours wrap periodically) */
static void derivs_at(const lattice *L, const double *X, size_t r, double grad[3], double *lap)
{
    const double cs2 = 1.0 / 3.0;
    double gx = 0, gy = 0, gz = 0, l = 0;
    const double x0 = X[r];
    for (int i = 1; i < L->Q; ++i) {
        const double xn = X[shift(L, r, i, +1)];
        gx += L->w[i] * L->e[i][0] * xn;
        gy += L->w[i] * L->e[i][1] * xn;
        gz += L->w[i] * L->e[i][2] * xn;
        l += L->w[i] * (xn - x0);
    }
    grad[0] = gx / cs2; grad[1] = gy / cs2; grad[2] = gz / cs2;
    *lap = 2.0 * l / cs2;
}

/* Derivatives of one field at every node.  grad is [3][N], lap is [N]. */
void orc_derivatives(const orc_params *p, const double *X, double *grad, double *lap)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return;
    const size_t N = L.N;
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        double gr[3], l;
        derivs_at(&L, X, (size_t)rr, gr, &l);
        for (int a = 0; a < 3; ++a) grad[(size_t)a * N + (size_t)rr] = gr[a];
        lap[rr] = l;
    }
}

/* ------------------------------------------ O3-O6 equilibria and collision */

/* Post-collision populations at every fluid node from moment arrays (with ghosts
 * already filled on solid nodes).  Solid nodes get zeros. */
static void collide_all(const orc_params *p, const lattice *L, const uint8_t *solid,
                        const double *f, const double *g, const double *k,
                        const double *rho, const double *jx, const double *jy, const double *jz,
                        const double *phi, const double *psi,
                        double *fs, double *gs, double *ks)
{
    const size_t N = L->N;
    const double *F[3] = {rho, phi, psi};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        if (is_solid(solid, r)) {
            for (int i = 0; i < L->Q; ++i) {
                fs[(size_t)i * N + r] = 0.0; gs[(size_t)i * N + r] = 0.0; ks[(size_t)i * N + r] = 0.0;
            }
            continue;
        }
        double X[3] = {rho[r], phi[r], psi[r]};
        double j[3] = {jx[r], jy[r], jz[r]};
        double grad[3][3], lap[3];
        for (int c = 0; c < 3; ++c) derivs_at(L, F[c], r, grad[c], &lap[c]);
        double feq[19], geq[19], keq[19];
        orc_equilibrium_node(p, X, j, (const double (*)[3])grad, lap, feq, geq, keq);
        for (int i = 0; i < L->Q; ++i) {
            const size_t o = (size_t)i * N + r;
            fs[o] = f[o] - (f[o] - feq[i]) / p->tau[0];
            gs[o] = g[o] - (g[o] - geq[i]) / p->tau[1];
            ks[o] = k[o] - (k[o] - keq[i]) / p->tau[2];
        }
    }
}

/* ------------------------------------------------------------- O7 stream */

/* Pull streaming with halfway bounce-back: x_i(r) <- x*_i(r - e_i) when that
 * node is fluid, else x*_{opp(i)}(r).  Solid nodes get zeros. */
void orc_stream(const orc_params *p, const uint8_t *solid, const double *xs, double *x)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return;
    const size_t N = L.N;
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        for (int i = 0; i < L.Q; ++i) {
            double v = 0.0;
            if (!is_solid(solid, r)) {
                const size_t src = shift(&L, r, i, -1);
                v = is_solid(solid, src) ? xs[(size_t)L.opp[i] * N + r] : xs[(size_t)i * N + src];
            }
            x[(size_t)i * N + r] = v;
        }
    }
}

/* ---------------------------------------------------------------- drivers */

typedef struct {
    double *rho, *jx, *jy, *jz, *phi, *psi, *fs, *gs, *ks;
} work;

static int work_alloc(work *w, size_t N, int Q)
{
    memset(w, 0, sizeof *w);
    w->rho = calloc(N, sizeof(double)); w->jx = calloc(N, sizeof(double));
    w->jy = calloc(N, sizeof(double));  w->jz = calloc(N, sizeof(double));
    w->phi = calloc(N, sizeof(double)); w->psi = calloc(N, sizeof(double));
    w->fs = calloc((size_t)Q * N, sizeof(double));
    w->gs = calloc((size_t)Q * N, sizeof(double));
    w->ks = calloc((size_t)Q * N, sizeof(double));
    return (w->rho && w->jx && w->jy && w->jz && w->phi && w->psi && w->fs && w->gs && w->ks) ? 0 : -1;
}

static void work_free(work *w)
{
    free(w->rho); free(w->jx); free(w->jy); free(w->jz); free(w->phi); free(w->psi);
    free(w->fs); free(w->gs); free(w->ks);
}

/* Advance conventional populations f, g, k ([Q][N] each) by nsteps time steps. */
int orc_step(const orc_params *p, const uint8_t *solid, double *f, double *g, double *k, long nsteps)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return -1;
    work w;
    if (work_alloc(&w, L.N, L.Q) != 0) { work_free(&w); return -2; }
    for (long t = 0; t < nsteps; ++t) {
        orc_moments(p, solid, f, g, k, w.rho, w.jx, w.jy, w.jz, w.phi, w.psi);   /* O1 */
        orc_ghosts(p, solid, w.rho, w.phi, w.psi);                                 /* O2 */
        collide_all(p, &L, solid, f, g, k, w.rho, w.jx, w.jy, w.jz, w.phi, w.psi,  /* O3-O6 */
                    w.fs, w.gs, w.ks);
        orc_stream(p, solid, w.fs, f);                                             /* O7 */
        orc_stream(p, solid, w.gs, g);
        orc_stream(p, solid, w.ks, k);
    }
    work_free(&w);
    return 0;
}

/* Populations at equilibrium with the given fields (velocity arrays may be NULL
 * for rest); derivatives use the same stencils and ghosts as a step. */
int orc_init_equilibrium(const orc_params *p, const uint8_t *solid, const double *rho,
                         const double *phi, const double *psi, const double *ux,
                         const double *uy, const double *uz, double *f, double *g, double *k)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return -1;
    const size_t N = L.N;
    work w;
    if (work_alloc(&w, N, L.Q) != 0) { work_free(&w); return -2; }
    for (size_t r = 0; r < N; ++r) {
        const int sld = is_solid(solid, r);
        w.rho[r] = sld ? 0.0 : rho[r];
        w.phi[r] = sld ? 0.0 : phi[r];
        w.psi[r] = sld ? 0.0 : psi[r];
        w.jx[r] = (sld || !ux) ? 0.0 : rho[r] * ux[r];
        w.jy[r] = (sld || !uy) ? 0.0 : rho[r] * uy[r];
        w.jz[r] = (sld || !uz) ? 0.0 : rho[r] * uz[r];
    }
    orc_ghosts(p, solid, w.rho, w.phi, w.psi);
    const double *F[3] = {w.rho, w.phi, w.psi};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        double feq[19], geq[19], keq[19];
        if (is_solid(solid, r)) {
            for (int i = 0; i < L.Q; ++i) feq[i] = geq[i] = keq[i] = 0.0;
        } else {
            double X[3] = {w.rho[r], w.phi[r], w.psi[r]};
            double j[3] = {w.jx[r], w.jy[r], w.jz[r]};
            double grad[3][3], lap[3];
            for (int c = 0; c < 3; ++c) derivs_at(&L, F[c], r, grad[c], &lap[c]);
            orc_equilibrium_node(p, X, j, (const double (*)[3])grad, lap, feq, geq, keq);
        }
        for (int i = 0; i < L.Q; ++i) {
            f[(size_t)i * N + r] = feq[i];
            g[(size_t)i * N + r] = geq[i];
            k[(size_t)i * N + r] = keq[i];
        }
    }
    work_free(&w);
    return 0;
}

/* O8: sums of rho, phi, psi over fluid nodes (Kahan, row-major order). */
void orc_mass(const orc_params *p, const uint8_t *solid, const double *f, const double *g,
              const double *k, double out[3])
{
    lattice L;
    if (lattice_init(&L, p) != 0) return;
    const size_t N = L.N;
    const double *P[3] = {f, g, k};
    for (int c = 0; c < 3; ++c) {
        double s = 0.0, comp = 0.0;
        for (size_t r = 0; r < N; ++r) {
            if (is_solid(solid, r)) continue;
            double v = 0.0;
            for (int i = 0; i < L.Q; ++i) v += P[c][(size_t)i * N + r];
            const double y = v - comp;
            const double t = s + y;
            comp = (t - s) - y;
            s = t;
        }
        out[c] = s;
    }
}

/* ---------------------------------------------------- forcing coupling (Guo) */

/* Chemical potentials (mu_rho, mu_phi, mu_psi) [3][N] of fields X at every node. */
static void chemical_potentials(const orc_params *p, const lattice *L, const double *rho, const double *phi,
                                const double *psi, double *mu)
{
    const size_t N = L->N;
    const double *F[3] = {rho, phi, psi};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        double X[3] = {rho[r], phi[r], psi[r]}, lap[3], gr[3], C[3], m[3], pb;
        for (int c = 0; c < 3; ++c) derivs_at(L, F[c], r, gr, &lap[c]);
        orc_thermo_node(p, X, lap, C, m, &pb);
        for (int c = 0; c < 3; ++c) mu[(size_t)c * N + r] = m[c];
    }
}

/* Non-ideal part of the pressure tensor, P_ab - rho c_s^2 delta_ab, at one node
 * (Sec. Equations of Motion, with the p_b, alpha^2 and cross-term readings of
 * the header), components xx yy zz xy yz zx. */
static void nonideal_pressure(const orc_params *p, const double X[3], const double grad[3][3],
                              const double lap[3], double Pi[6])
{
    const double a2 = p->alpha * p->alpha;
    double C[3], mu[3], pb;
    orc_thermo_node(p, X, lap, C, mu, &pb);
    double K[3][3];
    mixing(p, K);
    static const int ca[6] = {0, 1, 2, 0, 1, 2};
    static const int cb[6] = {0, 1, 2, 1, 2, 0};
    /* isotropic part: p_b - rho/3 - alpha^2 [sum_X K_XX (|grad X|^2 / 2 + X lap X)
     *   + sum_{X<Y} K_XY (grad X . grad Y + X lap Y + Y lap X)] */
    double iso = pb - X[0] / 3.0;
    for (int x = 0; x < 3; ++x) {
        const double g2 = grad[x][0] * grad[x][0] + grad[x][1] * grad[x][1] + grad[x][2] * grad[x][2];
        iso -= a2 * K[x][x] * (0.5 * g2 + X[x] * lap[x]);
        for (int y = x + 1; y < 3; ++y) {
            const double gg = grad[x][0] * grad[y][0] + grad[x][1] * grad[y][1] + grad[x][2] * grad[y][2];
            iso -= a2 * K[x][y] * (gg + X[x] * lap[y] + X[y] * lap[x]);
        }
    }
    for (int c = 0; c < 6; ++c) {
        const int al = ca[c], be = cb[c];
        double s = 0.0;
        for (int x = 0; x < 3; ++x) {
            s += K[x][x] * grad[x][al] * grad[x][be];
            for (int y = x + 1; y < 3; ++y) s += K[x][y] * (grad[x][al] * grad[y][be] + grad[y][al] * grad[x][be]);
        }
        Pi[c] = a2 * s + (c < 3 ? iso : 0.0);
    }
}

/* Body force F [3][N] = -div (P - rho c_s^2 I) of the fields rho, phi, psi
 * (periodic lattice). */
static void force_field(const orc_params *p, const lattice *L, const double *rho, const double *phi,
                        const double *psi, double *Pi, double *F)
{
    const size_t N = L->N;
    const double *X3[3] = {rho, phi, psi};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        double X[3] = {rho[r], phi[r], psi[r]}, grad[3][3], lap[3], P6[6];
        for (int c = 0; c < 3; ++c) derivs_at(L, X3[c], r, grad[c], &lap[c]);
        nonideal_pressure(p, X, (const double (*)[3])grad, lap, P6);
        for (int c = 0; c < 6; ++c) Pi[(size_t)c * N + r] = P6[c];
    }
    /* component (a, b) of the symmetric tensor in the xx yy zz xy yz zx order */
    static const int comp[3][3] = {{0, 3, 5}, {3, 1, 4}, {5, 4, 2}};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        for (int a = 0; a < 3; ++a) {
            double div = 0.0;
            for (int b = 0; b < 3; ++b) {
                double gb[3], lb;
                derivs_at(L, Pi + (size_t)comp[a][b] * N, r, gb, &lb);
                div += gb[b];
            }
            F[(size_t)a * N + r] = -div;
        }
    }
}

int orc_force(const orc_params *p, const double *rho, const double *phi, const double *psi, double *F)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return -1;
    double *Pi = calloc(6 * L.N, sizeof(double));
    if (!Pi) return -2;
    force_field(p, &L, rho, phi, psi, Pi, F);
    free(Pi);
    return 0;
}

/* Equilibria of the forcing coupling at one node: ideal-gas f_eq at velocity u,
 * g_eq and k_eq with mu_phi, mu_psi; directions i >= 1 from the formulas, i = 0
 * from the mass constraints. */
static void equilibrium_guo(const orc_params *p, const lattice *L, const double X[3], const double u[3],
                            const double mu[3], double *feq, double *geq, double *keq)
{
    const double cs2 = 1.0 / 3.0;
    const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double sf = 0.0, sg = 0.0, sk = 0.0;
    for (int i = 1; i < L->Q; ++i) {
        double eu = 0.0;
        for (int a = 0; a < 3; ++a) eu += L->e[i][a] * u[a];
        const double quad = (eu * eu - cs2 * uu) / (2.0 * cs2 * cs2);
        const double wi = L->w[i];
        feq[i] = wi * X[0] * (1.0 + eu / cs2 + quad);
        geq[i] = wi * (p->gamma[0] * mu[1] / cs2 + X[1] * eu / cs2 + X[1] * quad);
        keq[i] = wi * (p->gamma[1] * mu[2] / cs2 + X[2] * eu / cs2 + X[2] * quad);
        sf += feq[i]; sg += geq[i]; sk += keq[i];
    }
    feq[0] = X[0] - sf;
    geq[0] = X[1] - sg;
    keq[0] = X[2] - sk;
}

/* Advance populations f, g, k ([Q][N] each, periodic lattice) by nsteps time
 * steps of the forcing coupling. */
int orc_step_guo(const orc_params *p, double *f, double *g, double *k, long nsteps)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return -1;
    const size_t N = L.N;
    work w;
    double *mu = calloc(3 * N, sizeof(double)), *Pi = calloc(6 * N, sizeof(double)),
           *F = calloc(3 * N, sizeof(double));
    if (work_alloc(&w, N, L.Q) != 0 || !mu || !Pi || !F) {
        work_free(&w); free(mu); free(Pi); free(F);
        return -2;
    }
    const double cs2 = 1.0 / 3.0;
    for (long t = 0; t < nsteps; ++t) {
        orc_moments(p, NULL, f, g, k, w.rho, w.jx, w.jy, w.jz, w.phi, w.psi);
        chemical_potentials(p, &L, w.rho, w.phi, w.psi, mu);
        force_field(p, &L, w.rho, w.phi, w.psi, Pi, F);
#pragma omp parallel for schedule(static)
        for (long rr = 0; rr < (long)N; ++rr) {
            const size_t r = (size_t)rr;
            const double X[3] = {w.rho[r], w.phi[r], w.psi[r]};
            const double m[3] = {mu[r], mu[N + r], mu[2 * N + r]};
            const double Fr[3] = {F[r], F[N + r], F[2 * N + r]};
            const double j[3] = {w.jx[r], w.jy[r], w.jz[r]};
            double u[3];
            for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * Fr[a]) / X[0];
            double feq[19], geq[19], keq[19];
            equilibrium_guo(p, &L, X, u, m, feq, geq, keq);
            const double pref = 1.0 - 1.0 / (2.0 * p->tau[0]);
            for (int i = 0; i < L.Q; ++i) {
                double eu = 0.0, eF = 0.0, uF = 0.0;
                for (int a = 0; a < 3; ++a) {
                    eu += L.e[i][a] * u[a];
                    eF += L.e[i][a] * Fr[a];
                    uF += u[a] * Fr[a];
                }
                const double Si = pref * L.w[i] * ((eF - uF) / cs2 + eu * eF / (cs2 * cs2));
                const size_t o = (size_t)i * N + r;
                w.fs[o] = f[o] - (f[o] - feq[i]) / p->tau[0] + Si;
                w.gs[o] = g[o] - (g[o] - geq[i]) / p->tau[1];
                w.ks[o] = k[o] - (k[o] - keq[i]) / p->tau[2];
            }
        }
        orc_stream(p, NULL, w.fs, f);
        orc_stream(p, NULL, w.gs, g);
        orc_stream(p, NULL, w.ks, k);
    }
    work_free(&w);
    free(mu); free(Pi); free(F);
    return 0;
}

/* Populations at the forcing coupling's equilibrium with the given fields at
 * rest (periodic lattice): f_eq at u = 0, g_eq and k_eq with mu. */
int orc_init_equilibrium_guo(const orc_params *p, const double *rho, const double *phi, const double *psi,
                             double *f, double *g, double *k)
{
    lattice L;
    if (lattice_init(&L, p) != 0) return -1;
    const size_t N = L.N;
    double *mu = calloc(3 * N, sizeof(double));
    if (!mu) return -2;
    chemical_potentials(p, &L, rho, phi, psi, mu);
    const double u0[3] = {0.0, 0.0, 0.0};
#pragma omp parallel for schedule(static)
    for (long rr = 0; rr < (long)N; ++rr) {
        const size_t r = (size_t)rr;
        const double X[3] = {rho[r], phi[r], psi[r]};
        const double m[3] = {mu[r], mu[N + r], mu[2 * N + r]};
        double feq[19], geq[19], keq[19];
        equilibrium_guo(p, &L, X, u0, m, feq, geq, keq);
        for (int i = 0; i < L.Q; ++i) {
            f[(size_t)i * N + r] = feq[i];
            g[(size_t)i * N + r] = geq[i];
            k[(size_t)i * N + r] = keq[i];
        }
    }
    free(mu);
    return 0;
}
