/*
 * fre_oracle.c -- plain FP64 CPU oracle of the two-lattice free energy LBM of
 * Simonis et al., arXiv:2212.01617.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests, by __graft_entry__.smoke()
 * and by bench.py's CPU-baseline leg; the product path never touches it.  It
 * shares no code with the CUDA library.  Built with -ffp-contract=off so
 * every operation is a single IEEE FP64 round-to-nearest operation.
 *
 * What one time step computes, in the paper's order (Sec. 2.2, Algorithm 1,
 * Sec. 2.3), for every fluid node x, from the pre-collision populations:
 *   1. rho = sum_i f_i  (Eq. densMoment),  phi = sum_i g_i  (Eq. ordeMoment)
 *   2. mu  = A(phi^3 - phi) - kappa lap(phi)
 *      (Eq. mu_phi with kappa_1 = kappa_2 and rho = 1; A = kappa_p/4,
 *       kappa = alpha^2 kappa_p / 2).  lap is the isotropic lattice stencil
 *       lap(phi)(x) = (2/cs^2) sum_i w_i (phi(x+c_i) - phi(x)).
 *   3. F   = -phi grad(mu)   (Eq. F with the rho grad(mu_rho) term dropped),
 *      written with the product rule as F = mu grad(phi) - grad(phi mu) and
 *      the isotropic lattice gradient grad(a)(x) = (1/cs^2) sum_i w_i c_i
 *      a(x+c_i).  (The literal lattice form -phi grad_h(mu) feeds the
 *      k = (pi,0) momentum mode that BGK leaves undamped and is unstable for
 *      a resting interface; the product-rule form is the same force in the
 *      continuum and damps that mode.)
 *   4. rho u = sum_i c_i f_i + F/2  (Eq. veloMoment)
 *   5. S_i  Guo forcing (Eq. Fi), f_eq (Eq. feq), BGK (Eq. bgk, Eq. LBE):
 *      f*_i = f_i - (f_i - f_eq_i)/tau_f + S_i
 *   6. g_eq (Eq. geq, g_eq_0 = phi - sum_{i!=0} g_eq_i), g*_i = g_i -
 *      (g_i - g_eq_i)/tau_g  (Eq. LBEg)
 *   7. streaming f(x+c_i, t+1) = f*(x, t)  (Sec. 2.3), with half-way
 *      bounce-back and the moving-wall term (the usual LBM boundary
 *      treatment the paper defers to, Sec. 2.3) where the source node x-c_i
 *      is solid:
 *         f_i(x,t+1) = f*_ibar(x,t) + 2 w_i rho_w (c_i . u_w) / cs^2,
 *         g_i(x,t+1) = g*_ibar(x,t) + 2 w_i phi(x,t) (c_i . u_w) / cs^2,
 *      with rho_w = rho0.
 * Readings of points the paper leaves open:
 *   - stencil values at solid nodes: flat shear walls mirror across the
 *     half-way wall (value of the fluid node at y=0 / y=ny-1); roller solids
 *     take the w-weighted mean of their fluid lattice neighbours;
 *   - devices: parallel-band shear (walls at y=-1/2 and y=ny-1/2 moving at
 *     -u_wall / +u_wall, periodic in x and z), four-roller (four staircase
 *     cylinders of radius nx/8 centred at ((nx-1)/2 +- nx/4, (ny-1)/2 +- ny/4),
 *     surface speed u_wall, top-right and bottom-left counter-clockwise, the
 *     other two clockwise, periodic outer box), fully periodic box.
 * The four-roller wall point of a link (x - c_i/2, taken in the frame of the
 * roller the link meets: a roller of a box with ny = nx/2 reaches across the
 * periodic y boundary, where the node's image beside it counts) and the
 * weighted-mean stencil rule at roller solids are readings that no closed
 * form fixes;
 * the tests recompute one step of them from the geometry alone (indices,
 * signs, points).  For a rigid rotation c_i . u_w does not depend on where
 * along the link the wall point sits (c_i . (z x c_i) = 0).
 *
 * Canonical direction order (also the exchange order of the populations):
 *   D2Q9 : 0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1); 5 (1,1); 6 (-1,1);
 *          7 (-1,-1); 8 (1,-1)
 *   D3Q19: 0 rest; 1 (1,0,0); 2 (-1,0,0); 3 (0,1,0); 4 (0,-1,0); 5 (0,0,1);
 *          6 (0,0,-1); 7 (1,1,0); 8 (-1,-1,0); 9 (1,0,1); 10 (-1,0,-1);
 *          11 (0,1,1); 12 (0,-1,-1); 13 (1,-1,0); 14 (-1,1,0); 15 (1,0,-1);
 *          16 (-1,0,1); 17 (0,1,-1); 18 (0,-1,1)
 */
#include "fre_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* lattice speed of sound squared, textbook value for D2Q9 and D3Q19 */
static const double CS2 = 1.0 / 3.0;

static const int C_D2Q9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
static const double W_D2Q9[9] = {
    4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

static const int C_D3Q19[19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, 0, 1}, {-1, 0, -1}, {0, 1, 1}, {0, -1, -1},
    {1, -1, 0}, {-1, 1, 0}, {1, 0, -1}, {-1, 0, 1}, {0, 1, -1}, {0, -1, 1}};
static const double W_D3Q19[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

struct orc_state {
    orc_params p;
    int q;
    const int (*c)[3];
    const double *w;
    int opp[19];
    long long n;
    double *f, *g;         /* pre-collision populations [q][n] */
    double *fs, *gs;       /* post-collision populations [q][n] */
    double *rho, *phi, *mu, *ux, *uy, *uz, *Fx, *Fy, *Fz;
    double *mu_rho;        /* full functional: mu_rho (mu holds mu_phi) */
    signed char *solid;    /* 0 fluid, k in 1..4: inside roller k */
    double rc[5][2];       /* roller centres (index 1..4) */
    double omega[5];       /* roller angular velocities, counter-clockwise > 0 */
    double rr;             /* roller radius */
    long long step;
};

/* ------------------------------------------------------------------ lattice */

static void set_lattice(int lattice, int *q, const int (**c)[3], const double **w)
{
    if (lattice == ORC_D2Q9) { *q = 9; *c = C_D2Q9; *w = W_D2Q9; }
    else { *q = 19; *c = C_D3Q19; *w = W_D3Q19; }
}

int orc_lattice_info(int lattice, int *q, int *c, double *w)
{
    int qq; const int (*cc)[3]; const double *ww;
    if (lattice != ORC_D2Q9 && lattice != ORC_D3Q19) return -1;
    set_lattice(lattice, &qq, &cc, &ww);
    *q = qq;
    for (int i = 0; i < qq; ++i) {
        if (c) for (int a = 0; a < 3; ++a) c[3 * i + a] = cc[i][a];
        if (w) w[i] = ww[i];
    }
    return 0;
}

/* Eq. feq: f_eq_i = w_i rho [1 + c_ia u_a/cs^2 + u_a u_b (c_ia c_ib - cs^2 d_ab)/(2 cs^4)] */
static void feq_node(int q, const int (*c)[3], const double *w, double rho,
                     const double u[3], double *out)
{
    for (int i = 0; i < q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += c[i][a] * u[a];
        double quad = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                quad += u[a] * u[b] * (c[i][a] * c[i][b] - (a == b ? CS2 : 0.0));
        out[i] = w[i] * rho * (1.0 + cu / CS2 + quad / (2.0 * CS2 * CS2));
    }
}

/* Eq. geq: for i != 0
 *   g_eq_i = w_i [Gamma mu / cs^2 + phi c_ia u_a / cs^2
 *                 + phi u_a u_b (c_ia c_ib - cs^2 d_ab) / (2 cs^4)],
 * and g_eq_0 = phi - sum_{i != 0} g_eq_i. */
static void geq_node(int q, const int (*c)[3], const double *w, double phi,
                     double mu, double Gamma, const double u[3], double *out)
{
    double rest = phi;
    for (int i = 1; i < q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += c[i][a] * u[a];
        double quad = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                quad += u[a] * u[b] * (c[i][a] * c[i][b] - (a == b ? CS2 : 0.0));
        out[i] = w[i] * (Gamma * mu / CS2 + phi * cu / CS2 + phi * quad / (2.0 * CS2 * CS2));
        rest -= out[i];
    }
    out[0] = rest;
}

/* Eq. Fi (Guo): S_i = (1 - 1/(2 tau)) w_i [(c_i - u)/cs^2 + (c_i . u) c_i / cs^4] . F */
static void guo_node(int q, const int (*c)[3], const double *w, double tau,
                     const double u[3], const double F[3], double *out)
{
    for (int i = 0; i < q; ++i) {
        double cu = 0.0;
        for (int a = 0; a < 3; ++a) cu += c[i][a] * u[a];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += ((c[i][a] - u[a]) / CS2 + cu * c[i][a] / (CS2 * CS2)) * F[a];
        out[i] = (1.0 - 1.0 / (2.0 * tau)) * w[i] * s;
    }
}

void orc_feq(int lattice, double rho, const double u[3], double *out)
{
    int q; const int (*c)[3]; const double *w;
    set_lattice(lattice, &q, &c, &w);
    feq_node(q, c, w, rho, u, out);
}

void orc_geq(int lattice, double phi, double mu, double Gamma, const double u[3], double *out)
{
    int q; const int (*c)[3]; const double *w;
    set_lattice(lattice, &q, &c, &w);
    geq_node(q, c, w, phi, mu, Gamma, u, out);
}

void orc_guo(int lattice, double tau, const double u[3], const double F[3], double *out)
{
    int q; const int (*c)[3]; const double *w;
    set_lattice(lattice, &q, &c, &w);
    guo_node(q, c, w, tau, u, F, out);
}

/* ----------------------------------------------------------------- geometry */

/* periodic wrap of a coordinate that is at most one period outside [0, n) */
static int wrap(int a, int n)
{
    if (a < 0) return a + n;
    if (a >= n) return a - n;
    return a;
}

static long long node(const orc_state *s, int x, int y, int z)
{
    return ((long long)z * s->p.ny + y) * s->p.nx + x;
}

static void coords(const orc_state *s, long long n, int *x, int *y, int *z)
{
    int nx = s->p.nx, ny = s->p.ny;
    int r = (int)(n % ((long long)nx * ny));
    *x = r % nx;
    *y = r / nx;
    *z = (int)(n / ((long long)nx * ny));
}

static int roller_of(const orc_state *s, int x, int y)
{
    for (int k = 1; k <= 4; ++k) {
        double dx = x - s->rc[k][0], dy = y - s->rc[k][1];
        if (dx * dx + dy * dy <= s->rr * s->rr) return k;
    }
    return 0;
}

int orc_is_solid(const orc_state *s, int x, int y, int z)
{
    return s->solid[node(s, x, y, z)] != 0;
}

/* Lattice neighbour x + c_i used by the Laplacian and gradient stencils.
 * Periodic in x and z; in y periodic except for the shear device, whose
 * value outside the channel is the mirror image across the half-way wall. */
static long long stencil_nb(const orc_state *s, int x, int y, int z, int i)
{
    int xn = wrap(x + s->c[i][0], s->p.nx);
    int zn = wrap(z + s->c[i][2], s->p.nz);
    int yn = y + s->c[i][1];
    if (s->p.device == ORC_SHEAR) {
        if (yn < 0) yn = 0;
        if (yn >= s->p.ny) yn = s->p.ny - 1;
    } else {
        yn = wrap(yn, s->p.ny);
    }
    return node(s, xn, yn, zn);
}

/* Streaming source x - c_i.  Returns 1 and the source node when it is fluid;
 * returns 0 and the wall velocity at the link's wall point x - c_i/2 when it
 * is solid. */
static int stream_source(const orc_state *s, int x, int y, int z, int i,
                         long long *src, double uw[3])
{
    int xs = x - s->c[i][0], ys = y - s->c[i][1], zs = z - s->c[i][2];
    uw[0] = uw[1] = uw[2] = 0.0;
    if (s->p.device == ORC_SHEAR) {
        if (ys < 0) { uw[0] = -s->p.u_wall; return 0; }
        if (ys >= s->p.ny) { uw[0] = s->p.u_wall; return 0; }
        *src = node(s, wrap(xs, s->p.nx), ys, wrap(zs, s->p.nz));
        return 1;
    }
    *src = node(s, wrap(xs, s->p.nx), wrap(ys, s->p.ny), wrap(zs, s->p.nz));
    int k = s->solid[*src];
    if (k == 0) return 1;
    /* rigid rotation of roller k about its axis (parallel to z), at the
     * link's wall point in the frame of the roller: the wrapped source plus
     * c_i / 2 (a roller of a box with ny = nx/2 reaches across the
     * periodic y boundary) */
    double xw = wrap(xs, s->p.nx) + 0.5 * s->c[i][0], yw = wrap(ys, s->p.ny) + 0.5 * s->c[i][1];
    uw[0] = -s->omega[k] * (yw - s->rc[k][1]);
    uw[1] = s->omega[k] * (xw - s->rc[k][0]);
    return 0;
}

/* Values of a stencil field at roller solids: w-weighted mean of the fluid
 * lattice neighbours (solids without fluid neighbours keep 0). */
static void fill_ghosts(orc_state *s, double *field)
{
    if (s->p.device != ORC_FOUR_ROLLER) return;
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (!s->solid[n]) continue;
        int x, y, z;
        coords(s, n, &x, &y, &z);
        double num = 0.0, den = 0.0;
        for (int j = 1; j < s->q; ++j) {
            long long m = stencil_nb(s, x, y, z, j);
            if (s->solid[m]) continue;
            num += s->w[j] * field[m];
            den += s->w[j];
        }
        field[n] = den > 0.0 ? num / den : 0.0;
    }
}

/* ------------------------------------------------------------ create/free */

orc_state *orc_create(const orc_params *p)
{
    if (!p) return NULL;
    if (p->lattice != ORC_D2Q9 && p->lattice != ORC_D3Q19) return NULL;
    if (p->device < ORC_SHEAR || p->device > ORC_PERIODIC) return NULL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return NULL;
    if (p->lattice == ORC_D2Q9 && p->nz != 1) return NULL;
    if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return NULL;
    if (p->model != 0 && p->model != 1) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    set_lattice(p->lattice, &s->q, &s->c, &s->w);
    for (int i = 0; i < s->q; ++i)
        for (int j = 0; j < s->q; ++j)
            if (s->c[j][0] == -s->c[i][0] && s->c[j][1] == -s->c[i][1] &&
                s->c[j][2] == -s->c[i][2])
                s->opp[i] = j;
    s->n = (long long)p->nx * p->ny * p->nz;
    size_t qn = (size_t)s->q * (size_t)s->n;
    s->f = calloc(qn, sizeof(double));
    s->g = calloc(qn, sizeof(double));
    s->fs = calloc(qn, sizeof(double));
    s->gs = calloc(qn, sizeof(double));
    double **fields[] = {&s->rho, &s->phi, &s->mu, &s->ux, &s->uy, &s->uz,
                         &s->Fx, &s->Fy, &s->Fz, &s->mu_rho};
    for (int k = 0; k < 10; ++k) *fields[k] = calloc((size_t)s->n, sizeof(double));
    s->solid = calloc((size_t)s->n, 1);
    int ok = s->f && s->g && s->fs && s->gs && s->solid;
    for (int k = 0; k < 10; ++k) ok = ok && *fields[k];
    if (!ok) { orc_destroy(s); return NULL; }
    if (p->device == ORC_FOUR_ROLLER) {
        double cx = 0.5 * (p->nx - 1), cy = 0.5 * (p->ny - 1);
        double ox = 0.25 * p->nx, oy = 0.25 * p->ny;
        s->rr = p->nx / 8.0;
        double om = p->u_wall / s->rr;
        s->rc[1][0] = cx + ox; s->rc[1][1] = cy + oy; s->omega[1] = om;   /* top right */
        s->rc[2][0] = cx - ox; s->rc[2][1] = cy + oy; s->omega[2] = -om;  /* top left */
        s->rc[3][0] = cx - ox; s->rc[3][1] = cy - oy; s->omega[3] = om;   /* bottom left */
        s->rc[4][0] = cx + ox; s->rc[4][1] = cy - oy; s->omega[4] = -om;  /* bottom right */
        for (long long n = 0; n < s->n; ++n) {
            int x, y, z;
            coords(s, n, &x, &y, &z);
            s->solid[n] = (signed char)roller_of(s, x, y);
        }
    }
    return s;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->f); free(s->g); free(s->fs); free(s->gs);
    free(s->rho); free(s->phi); free(s->mu); free(s->ux); free(s->uy); free(s->uz);
    free(s->Fx); free(s->Fy); free(s->Fz); free(s->mu_rho);
    free(s->solid);
    free(s);
}

int orc_q(const orc_state *s) { return s->q; }
long long orc_nodes(const orc_state *s) { return s->n; }

/* ------------------------------------------------------ macroscopic fields */

/* isotropic Laplacian of a field at fluid node n (ghosts filled) */
static double laplacian(const orc_state *s, const double *a, long long n)
{
    int x, y, z;
    coords(s, n, &x, &y, &z);
    double lap = 0.0;
    for (int i = 1; i < s->q; ++i)
        lap += s->w[i] * (a[stencil_nb(s, x, y, z, i)] - a[n]);
    return lap * (2.0 / CS2);
}

/* Step 2: mu at fluid nodes from phi (phi ghosts must be filled).
 * Reduced functional (model 0): mu = A(phi^3 - phi) - kappa lap(phi).
 * Full functional (model 1, Eq. mu_rho and Eq. mu_phi; rho ghosts filled
 * too), with a = rho + phi, b = rho - phi:
 *   mu_rho = k1/8 a(a-2)(a-1) + k2/8 b(b-2)(b-1)
 *            + alpha^2/4 [-(k1 + k2) lap(rho) + (k2 - k1) lap(phi)],
 *   mu_phi = k1/8 a(a-2)(a-1) - k2/8 b(b-2)(b-1)
 *            + alpha^2/4 [-(k1 + k2) lap(phi) + (k2 - k1) lap(rho)]. */
static void compute_mu(orc_state *s)
{
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) continue;
        double ph = s->phi[n];
        double lphi = laplacian(s, s->phi, n);
        if (s->p.model == 0) {
            s->mu[n] = s->p.A * (ph * ph * ph - ph) - s->p.kappa * lphi;
            continue;
        }
        double lrho = laplacian(s, s->rho, n);
        double k1 = s->p.kappa1, k2 = s->p.kappa2, al2 = s->p.alpha * s->p.alpha;
        double a = s->rho[n] + ph, b = s->rho[n] - ph;
        double ta = k1 / 8.0 * a * (a - 2.0) * (a - 1.0);
        double tb = k2 / 8.0 * b * (b - 2.0) * (b - 1.0);
        s->mu_rho[n] = ta + tb + al2 / 4.0 * (-(k1 + k2) * lrho + (k2 - k1) * lphi);
        s->mu[n] = ta - tb + al2 / 4.0 * (-(k1 + k2) * lphi + (k2 - k1) * lrho);
    }
    fill_ghosts(s, s->mu);
    if (s->p.model == 1) fill_ghosts(s, s->mu_rho);
}

/* Steps 1-4 from the pre-collision populations: rho, phi, mu, F, u. */
static void macro(orc_state *s)
{
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) { s->rho[n] = s->phi[n] = 0.0; continue; }
        double r = 0.0, ph = 0.0;
        for (int i = 0; i < s->q; ++i) {
            r += s->f[(size_t)i * s->n + n];
            ph += s->g[(size_t)i * s->n + n];
        }
        s->rho[n] = r;
        s->phi[n] = ph;
    }
    fill_ghosts(s, s->phi);
    if (s->p.model == 1) fill_ghosts(s, s->rho);
    compute_mu(s);
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) {
            s->ux[n] = s->uy[n] = s->uz[n] = 0.0;
            s->Fx[n] = s->Fy[n] = s->Fz[n] = 0.0;
            continue;
        }
        int x, y, z;
        coords(s, n, &x, &y, &z);
        /* grad(phi) and grad(phi mu) with the isotropic lattice gradient */
        double gp[3] = {0.0, 0.0, 0.0}, gpm[3] = {0.0, 0.0, 0.0};
        double gr[3] = {0.0, 0.0, 0.0}, grm[3] = {0.0, 0.0, 0.0};
        for (int i = 1; i < s->q; ++i) {
            long long m = stencil_nb(s, x, y, z, i);
            for (int a = 0; a < 3; ++a) {
                gp[a] += s->w[i] * s->c[i][a] * s->phi[m];
                gpm[a] += s->w[i] * s->c[i][a] * (s->phi[m] * s->mu[m]);
                if (s->p.model == 1) {
                    gr[a] += s->w[i] * s->c[i][a] * s->rho[m];
                    grm[a] += s->w[i] * s->c[i][a] * (s->rho[m] * s->mu_rho[m]);
                }
            }
        }
        /* F = -phi grad(mu) = mu grad(phi) - grad(phi mu); the full
         * functional adds -rho grad(mu_rho) = mu_rho grad(rho) - grad(rho mu_rho) */
        double F[3], j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < 3; ++a) {
            F[a] = s->mu[n] * (gp[a] / CS2) - gpm[a] / CS2;
            if (s->p.model == 1) F[a] += s->mu_rho[n] * (gr[a] / CS2) - grm[a] / CS2;
        }
        for (int i = 0; i < s->q; ++i) {
            double fi = s->f[(size_t)i * s->n + n];
            for (int a = 0; a < 3; ++a) j[a] += s->c[i][a] * fi;
        }
        s->Fx[n] = F[0]; s->Fy[n] = F[1]; s->Fz[n] = F[2];
        s->ux[n] = (j[0] + 0.5 * F[0]) / s->rho[n];
        s->uy[n] = (j[1] + 0.5 * F[1]) / s->rho[n];
        s->uz[n] = (j[2] + 0.5 * F[2]) / s->rho[n];
    }
}

/* ------------------------------------------------------------------- step */

static void collide(orc_state *s)
{
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) continue;
        double u[3] = {s->ux[n], s->uy[n], s->uz[n]};
        double F[3] = {s->Fx[n], s->Fy[n], s->Fz[n]};
        double feq[19], S[19], geq[19];
        feq_node(s->q, s->c, s->w, s->rho[n], u, feq);
        guo_node(s->q, s->c, s->w, s->p.tau_f, u, F, S);
        geq_node(s->q, s->c, s->w, s->phi[n], s->mu[n], s->p.Gamma, u, geq);
        for (int i = 0; i < s->q; ++i) {
            size_t k = (size_t)i * s->n + n;
            s->fs[k] = s->f[k] - (s->f[k] - feq[i]) / s->p.tau_f + S[i];
            s->gs[k] = s->g[k] - (s->g[k] - geq[i]) / s->p.tau_g;
        }
    }
}

/* Fraction q in (0, 1] of the link from fluid node (x, y) toward its solid
 * source (x, y) - c_i at which it crosses the surface of roller k (circle
 * of radius rr about rc[k]), measured from the fluid node.  The source's
 * wrapped coordinates place the circle; the fluid node is the source plus
 * c_i. */
static double link_fraction(const orc_state *s, int x, int y, int i, int k)
{
    int xs = wrap(x - s->c[i][0], s->p.nx), ys = wrap(y - s->c[i][1], s->p.ny);
    double dx = xs + s->c[i][0] - s->rc[k][0], dy = ys + s->c[i][1] - s->rc[k][1];
    double cx = s->c[i][0], cy = s->c[i][1];
    double cc = cx * cx + cy * cy, dc = dx * cx + dy * cy, dd = dx * dx + dy * dy - s->rr * s->rr;
    double disc = dc * dc - cc * dd;
    double t = (dc - sqrt(disc > 0.0 ? disc : 0.0)) / cc; /* first crossing of |d - t c| = r */
    if (t <= 0.0) t = 1e-12;
    if (t > 1.0) t = 1.0;
    return t;
}

static void stream(orc_state *s)
{
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) continue;
        int x, y, z;
        coords(s, n, &x, &y, &z);
        for (int i = 0; i < s->q; ++i) {
            long long src;
            double uw[3];
            size_t k = (size_t)i * s->n + n;
            if (stream_source(s, x, y, z, i, &src, uw)) {
                s->f[k] = s->fs[(size_t)i * s->n + src];
                s->g[k] = s->gs[(size_t)i * s->n + src];
            } else {
                double cu = 0.0;
                for (int a = 0; a < 3; ++a) cu += s->c[i][a] * uw[a];
                size_t kb = (size_t)s->opp[i] * s->n + n;
                double lf = 2.0 * s->w[i] * s->p.rho0 * cu / CS2, lg = 2.0 * s->w[i] * s->phi[n] * cu / CS2;
                if (s->p.interp && s->p.device == ORC_FOUR_ROLLER) {
                    /* interpolated bounce-back (linear, after Bouzidi et al.):
                     * the wall sits at x - q c_i; q < 1/2 interpolates the
                     * opposite population between x and x + c_i before it
                     * is reflected, q >= 1/2 between the reflected one and
                     * the node's own population i; the moving-wall term
                     * takes the matching weight (1 for q < 1/2, 1/(2q)) */
                    long long src2 = node(s, wrap(x - s->c[i][0], s->p.nx), wrap(y - s->c[i][1], s->p.ny),
                                          wrap(z - s->c[i][2], s->p.nz));
                    int kr = s->solid[src2];
                    double q = link_fraction(s, x, y, i, kr);
                    /* the wall velocity at the wall point x - q c_i itself */
                    double xw = wrap(x - s->c[i][0], s->p.nx) + (1.0 - q) * s->c[i][0];
                    double yw = wrap(y - s->c[i][1], s->p.ny) + (1.0 - q) * s->c[i][1];
                    cu = s->omega[kr] * (-(yw - s->rc[kr][1]) * s->c[i][0] + (xw - s->rc[kr][0]) * s->c[i][1]);
                    lf = 2.0 * s->w[i] * s->p.rho0 * cu / CS2;
                    lg = 2.0 * s->w[i] * s->phi[n] * cu / CS2;
                    long long m = node(s, wrap(x + s->c[i][0], s->p.nx), wrap(y + s->c[i][1], s->p.ny),
                                       wrap(z + s->c[i][2], s->p.nz));
                    if (q < 0.5 && !s->solid[m]) {
                        size_t km = (size_t)s->opp[i] * s->n + m;
                        s->f[k] = 2.0 * q * s->fs[kb] + (1.0 - 2.0 * q) * s->fs[km] + lf;
                        s->g[k] = 2.0 * q * s->gs[kb] + (1.0 - 2.0 * q) * s->gs[km] + lg;
                    } else if (q >= 0.5) {
                        size_t ki = (size_t)i * s->n + n;
                        s->f[k] = (s->fs[kb] + (2.0 * q - 1.0) * s->fs[ki] + lf) / (2.0 * q);
                        s->g[k] = (s->gs[kb] + (2.0 * q - 1.0) * s->gs[ki] + lg) / (2.0 * q);
                    } else {
                        /* no fluid node behind x: half-way bounce-back */
                        s->f[k] = s->fs[kb] + lf;
                        s->g[k] = s->gs[kb] + lg;
                    }
                } else {
                    s->f[k] = s->fs[kb] + lf;
                    s->g[k] = s->gs[kb] + lg;
                }
            }
        }
    }
}

int orc_step(orc_state *s, int nsteps)
{
    if (!s || nsteps < 0) return -1;
    for (int t = 0; t < nsteps; ++t) {
        macro(s);
        collide(s);
        stream(s);
        s->step++;
    }
    return 0;
}

/* --------------------------------------------------------- initialisation */

/* Populations at equilibrium for given rho, u, phi at the fluid nodes (the
 * equilibrium part of the initialisation of Sec. 2.3); mu follows from phi. */
static void init_equilibrium(orc_state *s)
{
    fill_ghosts(s, s->phi);
    if (s->p.model == 1) fill_ghosts(s, s->rho);
    compute_mu(s);
    #pragma omp parallel for schedule(static)
    for (long long n = 0; n < s->n; ++n) {
        double feq[19], geq[19];
        if (s->solid[n]) {
            for (int i = 0; i < s->q; ++i)
                s->f[(size_t)i * s->n + n] = s->g[(size_t)i * s->n + n] = 0.0;
            continue;
        }
        double u[3] = {s->ux[n], s->uy[n], s->uz[n]};
        feq_node(s->q, s->c, s->w, s->rho[n], u, feq);
        geq_node(s->q, s->c, s->w, s->phi[n], s->mu[n], s->p.Gamma, u, geq);
        for (int i = 0; i < s->q; ++i) {
            s->f[(size_t)i * s->n + n] = feq[i];
            s->g[(size_t)i * s->n + n] = geq[i];
        }
    }
    s->step = 0;
}

int orc_init_fields(orc_state *s, const double *rho, const double *ux,
                    const double *uy, const double *uz, const double *phi)
{
    if (!s || !rho || !ux || !uy || !phi) return -1;
    for (long long n = 0; n < s->n; ++n) {
        int fl = !s->solid[n];
        s->rho[n] = fl ? rho[n] : 0.0;
        s->ux[n] = fl ? ux[n] : 0.0;
        s->uy[n] = fl ? uy[n] : 0.0;
        s->uz[n] = (fl && uz) ? uz[n] : 0.0;
        s->phi[n] = fl ? phi[n] : 0.0;
    }
    init_equilibrium(s);
    return 0;
}

/* Droplet phi = tanh((R - |x - c|) / (sqrt(2) xi)), xi = sqrt(kappa/A), the
 * planar interface profile of Sec. 2.2 applied radially; rho = rho0; u is the
 * Couette profile of the moving walls for the shear device, 0 otherwise. */
int orc_init_droplet(orc_state *s, double cx, double cy, double cz, double R)
{
    if (!s || !(R > 0.0)) return -1;
    /* interface width: tanh(x / (sqrt(2) xi)) with xi = sqrt(kappa / A); the
     * full functional's planar profile is tanh(x / (2 alpha)), xi = sqrt(2)
     * alpha (each component's profile has width 2 alpha, whatever kappa_k) */
    double xi;
    if (s->p.model == 0) {
        if (!(s->p.A > 0.0) || !(s->p.kappa > 0.0)) return -1;
        xi = sqrt(s->p.kappa / s->p.A);
    } else {
        if (!(s->p.alpha > 0.0)) return -1;
        xi = sqrt(2.0) * s->p.alpha;
    }
    for (long long n = 0; n < s->n; ++n) {
        int x, y, z;
        coords(s, n, &x, &y, &z);
        double dx = x - cx, dy = y - cy, dz = (s->p.lattice == ORC_D3Q19) ? z - cz : 0.0;
        double r = sqrt(dx * dx + dy * dy + dz * dz);
        int fl = !s->solid[n];
        s->phi[n] = fl ? tanh((R - r) / (sqrt(2.0) * xi)) : 0.0;
        s->rho[n] = fl ? s->p.rho0 : 0.0;
        s->ux[n] = (fl && s->p.device == ORC_SHEAR)
                       ? s->p.u_wall * (2.0 * (y + 0.5) / s->p.ny - 1.0) : 0.0;
        s->uy[n] = 0.0;
        s->uz[n] = 0.0;
    }
    init_equilibrium(s);
    return 0;
}

int orc_load_populations(orc_state *s, const double *f, const double *g)
{
    if (!s || !f || !g) return -1;
    size_t qn = (size_t)s->q * s->n;
    for (size_t k = 0; k < qn; ++k) {
        int fl = !s->solid[k % (size_t)s->n];
        s->f[k] = fl ? f[k] : 0.0;
        s->g[k] = fl ? g[k] : 0.0;
    }
    s->step = 0;
    return 0;
}

int orc_store_populations(const orc_state *s, double *f, double *g)
{
    if (!s) return -1;
    size_t qn = (size_t)s->q * s->n;
    if (f) memcpy(f, s->f, qn * sizeof(double));
    if (g) memcpy(g, s->g, qn * sizeof(double));
    return 0;
}

int orc_fields(orc_state *s, double *rho, double *ux, double *uy, double *uz,
               double *phi, double *mu)
{
    if (!s) return -1;
    macro(s);
    for (long long n = 0; n < s->n; ++n) {
        int fl = !s->solid[n];
        if (rho) rho[n] = fl ? s->rho[n] : 0.0;
        if (ux) ux[n] = fl ? s->ux[n] : 0.0;
        if (uy) uy[n] = fl ? s->uy[n] : 0.0;
        if (uz) uz[n] = fl ? s->uz[n] : 0.0;
        if (phi) phi[n] = fl ? s->phi[n] : 0.0;
        if (mu) mu[n] = fl ? s->mu[n] : 0.0;
    }
    return 0;
}

/* ------------------------------------------------------------- observables */

typedef struct { double s, c; } nsum;  /* Neumaier compensated sum */

static void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

static double nval(const nsum *a) { return a->s + a->c; }

static double pressure(const orc_state *s, long long n)
{
    /* bulk thermodynamic pressure cs^2 rho + phi mu - psi(phi) with
     * psi = (A/4)(phi^2-1)^2, the bulk part of the reduced functional; the
     * full functional: cs^2 rho + rho mu_rho + phi mu_phi - psi(rho, phi),
     * psi = k1/32 a^2 (a-2)^2 + k2/32 b^2 (b-2)^2, a = rho + phi, b = rho - phi */
    double ph = s->phi[n];
    if (s->p.model == 1) {
        double a = s->rho[n] + ph, b = s->rho[n] - ph;
        double psi = s->p.kappa1 / 32.0 * a * a * (a - 2.0) * (a - 2.0) +
                     s->p.kappa2 / 32.0 * b * b * (b - 2.0) * (b - 2.0);
        return CS2 * s->rho[n] + s->rho[n] * s->mu_rho[n] + ph * s->mu[n] - psi;
    }
    double psi = 0.25 * s->p.A * (ph * ph - 1.0) * (ph * ph - 1.0);
    return CS2 * s->rho[n] + ph * s->mu[n] - psi;
}

/* Pressure at the point (X, Y, Z) by trilinear interpolation of the nodal
 * pressure: periodic in x and z, and in y off the shear device (whose y is
 * clamped to the fluid rows); solid nodes carry no weight.  The Laplace
 * law (Sec. 3) compares the pressure inside and outside a droplet; read at
 * the node nearest the centroid, a droplet centred on a cell face would
 * switch nodes under any rounding of its centroid. */
static double pressure_interp(const orc_state *s, double X, double Y, double Z)
{
    int x0 = (int)floor(X), y0 = (int)floor(Y), z0 = (int)floor(Z);
    double fx = X - x0, fy = Y - y0, fz = Z - z0;
    double acc = 0.0, wsum = 0.0;
    for (int k = 0; k < 8; ++k) {
        int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        double w = (dx ? fx : 1.0 - fx) * (dy ? fy : 1.0 - fy) * (dz ? fz : 1.0 - fz);
        if (w == 0.0) continue;
        int x = wrap(x0 + dx, s->p.nx), z = wrap(z0 + dz, s->p.nz), y = y0 + dy;
        if (s->p.device == ORC_SHEAR) {
            if (y < 0) y = 0;
            if (y >= s->p.ny) y = s->p.ny - 1;
        } else {
            y = wrap(y, s->p.ny);
        }
        long long n = node(s, x, y, z);
        if (s->solid[n]) continue;
        acc += w * pressure(s, n);
        wsum += w;
    }
    return wsum > 0.0 ? acc / wsum : 0.0;
}

int orc_observables(orc_state *s, orc_obs *o)
{
    if (!s || !o) return -1;
    memset(o, 0, sizeof(*o));
    macro(s);
    nsum mass = {0, 0}, phis = {0, 0}, vol = {0, 0}, W = {0, 0}, cnt = {0, 0};
    nsum mx = {0, 0}, my = {0, 0}, mz = {0, 0};
    int bad = 0;
    double umax = 0.0;
    for (long long n = 0; n < s->n; ++n) {
        if (s->solid[n]) continue;
        int x, y, z;
        coords(s, n, &x, &y, &z);
        double ph = s->phi[n];
        nadd(&mass, s->rho[n]);
        nadd(&phis, ph);
        nadd(&vol, 0.5 * (1.0 + ph));
        double u2 = s->ux[n] * s->ux[n] + s->uy[n] * s->uy[n] + s->uz[n] * s->uz[n];
        if (!isfinite(s->rho[n]) || !isfinite(ph) || !isfinite(u2) || !isfinite(s->mu[n])) bad = 1;
        else if (sqrt(u2) > umax) umax = sqrt(u2);
        if (ph > 0.0) {
            double wgt = 0.5 * (1.0 + ph);
            nadd(&W, wgt);
            nadd(&cnt, 1.0);
            nadd(&mx, wgt * x);
            nadd(&my, wgt * y);
            nadd(&mz, wgt * z);
        }
    }
    o->mass = nval(&mass);
    o->phi_sum = nval(&phis);
    o->volume = nval(&vol);
    o->drop_weight = nval(&W);
    o->drop_count = nval(&cnt);
    o->max_u = umax;
    o->step = s->step;
    if (o->drop_weight > 0.0) {
        double X[3] = {nval(&mx) / o->drop_weight, nval(&my) / o->drop_weight,
                       nval(&mz) / o->drop_weight};
        nsum I[6];
        memset(I, 0, sizeof(I));
        for (long long n = 0; n < s->n; ++n) {
            if (s->solid[n] || !(s->phi[n] > 0.0)) continue;
            int x, y, z;
            coords(s, n, &x, &y, &z);
            double wgt = 0.5 * (1.0 + s->phi[n]);
            double d[3] = {x - X[0], y - X[1], z - X[2]};
            nadd(&I[0], wgt * d[0] * d[0]);
            nadd(&I[1], wgt * d[1] * d[1]);
            nadd(&I[2], wgt * d[2] * d[2]);
            nadd(&I[3], wgt * d[0] * d[1]);
            nadd(&I[4], wgt * d[0] * d[2]);
            nadd(&I[5], wgt * d[1] * d[2]);
        }
        for (int k = 0; k < 3; ++k) o->centroid[k] = X[k];
        for (int k = 0; k < 6; ++k) o->I[k] = nval(&I[k]) / o->drop_weight;
        /* in-plane (x-y) ellipse of the second moments: L/B = sqrt(l1/l2) */
        double a = o->I[0], b = o->I[1], c = o->I[3];
        double m = 0.5 * (a + b), r = sqrt(0.25 * (a - b) * (a - b) + c * c);
        double l1 = m + r, l2 = m - r;
        if (l2 < 0.0) l2 = 0.0;
        double s1 = sqrt(l1), s2 = sqrt(l2);
        o->D = (s1 + s2) > 0.0 ? (s1 - s2) / (s1 + s2) : 0.0;
        o->theta_deg = 0.5 * atan2(2.0 * c, a - b) * 180.0 / M_PI;
        /* Laplace pressure: the pressure at the centroid vs the pressure
         * half a period away in x (and z) */
        o->p_centre = pressure_interp(s, X[0], X[1], X[2]);
        o->p_far = pressure_interp(s, X[0] + s->p.nx / 2, X[1], s->p.nz > 1 ? X[2] + s->p.nz / 2 : X[2]);
        o->dp = o->p_centre - o->p_far;
    }
    o->status = bad ? 1 : (umax > 0.3 ? 2 : 0);
    return 0;
}

/* ------------------------------------------- consistent initialisation */

/* Consistent initial populations (Sec. 2.3: the populations start at their
 * equilibrium and their kinetic moments are aligned by collisions before the
 * simulated time begins; the reference there is Mei et al. 2006).  Reading:
 * from the current pre-collision state (normally right after an
 * initialisation), take u0 = sum c_i f_i / rho, phi0 = sum g_i, mu0 and the
 * force F0 = mu0 grad(phi0) - grad(phi0 mu0) as they stand, then run
 * `iterations` collide-and-stream passes of f alone in which the velocity
 * of f_eq and of the Guo term is held at u0 and the force at F0, while the
 * density rho = sum f_i is free: the pressure field and the non-equilibrium
 * parts of f settle to what the flow and the interfacial force need.  The
 * order-parameter lattice ends at g = g_eq(phi0, mu0, u0).  The result is
 * the pre-collision state of step 0. */
int orc_init_consistent(orc_state *s, int iterations)
{
    if (!s || iterations < 0) return -1;
    const long long n = s->n;
    const int q = s->q;
    double *u0 = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!u0) return -1;
    macro(s); /* phi0 (ghosts), mu0 (ghosts), F0 */
    #pragma omp parallel for schedule(static)
    for (long long k = 0; k < n; ++k) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        if (!s->solid[k]) {
            for (int i = 0; i < q; ++i) {
                double fi = s->f[(size_t)i * n + k];
                r += fi;
                for (int a = 0; a < 3; ++a) j[a] += s->c[i][a] * fi;
            }
        }
        for (int a = 0; a < 3; ++a) u0[3 * k + a] = r != 0.0 ? j[a] / r : 0.0;
    }
    for (int it = 0; it < iterations; ++it) {
        /* collide f with u0 and F0 held */
        #pragma omp parallel for schedule(static)
        for (long long k = 0; k < n; ++k) {
            if (s->solid[k]) continue;
            double r = 0.0, feq[19], S[19];
            for (int i = 0; i < q; ++i) r += s->f[(size_t)i * n + k];
            double F[3] = {s->Fx[k], s->Fy[k], s->Fz[k]};
            feq_node(q, s->c, s->w, r, &u0[3 * k], feq);
            guo_node(q, s->c, s->w, s->p.tau_f, &u0[3 * k], F, S);
            for (int i = 0; i < q; ++i) {
                size_t m = (size_t)i * n + k;
                s->fs[m] = s->f[m] - (s->f[m] - feq[i]) / s->p.tau_f + S[i];
            }
        }
        /* stream f with the wall rule of the time step */
        #pragma omp parallel for schedule(static)
        for (long long k = 0; k < n; ++k) {
            if (s->solid[k]) continue;
            int x, y, z;
            coords(s, k, &x, &y, &z);
            for (int i = 0; i < q; ++i) {
                long long src;
                double uw[3];
                if (stream_source(s, x, y, z, i, &src, uw)) {
                    s->f[(size_t)i * n + k] = s->fs[(size_t)i * n + src];
                } else {
                    double cu = 0.0;
                    for (int a = 0; a < 3; ++a) cu += s->c[i][a] * uw[a];
                    s->f[(size_t)i * n + k] = s->fs[(size_t)s->opp[i] * n + k] + 2.0 * s->w[i] * s->p.rho0 * cu / CS2;
                }
            }
        }
    }
    /* g at the equilibrium of phi0, mu0 and u0 */
    #pragma omp parallel for schedule(static)
    for (long long k = 0; k < n; ++k) {
        if (s->solid[k]) continue;
        double geq[19];
        geq_node(q, s->c, s->w, s->phi[k], s->mu[k], s->p.Gamma, &u0[3 * k], geq);
        for (int i = 0; i < q; ++i) s->g[(size_t)i * n + k] = geq[i];
    }
    free(u0);
    s->step = 0;
    return 0;
}

/* ---------------------------------------------------- droplet components */

/* Connected components of the droplet phase, for breakup detection (Sec. 3:
 * a drop that breaks up leaves two or more separate drops).  The phase is
 * the set of fluid nodes with phi > 0 (phi = +1 inside the droplet).  Two
 * nodes of the phase are connected when a lattice velocity links them
 * (D2Q9: the 8 neighbours, D3Q19: the 18), with the device's periodic wrap:
 * x and z always, y except across the shear walls.  labels[n] = -1 outside
 * the phase, else the smallest node index of n's component.  A plain
 * breadth-first flood fill started from each unvisited phase node in
 * increasing index order, so the start node is its component's smallest
 * index.  Returns the number of components (-1 if out of memory). */
int orc_label_phase(const orc_state *s, const double *phi, int *labels)
{
    const long long n = s->n;
    long long *queue = (long long *)malloc((size_t)(n > 0 ? n : 1) * sizeof(long long));
    if (!queue) return -1;
    for (long long k = 0; k < n; ++k)
        labels[k] = (!s->solid[k] && phi[k] > 0.0) ? -2 : -1; /* -2: not yet visited */
    int count = 0;
    for (long long start = 0; start < n; ++start) {
        if (labels[start] != -2) continue;
        ++count;
        long long head = 0, tail = 0;
        queue[tail++] = start;
        labels[start] = (int)start;
        while (head < tail) {
            long long m = queue[head++];
            int x, y, z;
            coords(s, m, &x, &y, &z);
            for (int i = 1; i < s->q; ++i) {
                int yn = y + s->c[i][1];
                if (s->p.device == ORC_SHEAR && (yn < 0 || yn >= s->p.ny)) continue;
                long long nb = node(s, wrap(x + s->c[i][0], s->p.nx), wrap(yn, s->p.ny),
                                    wrap(z + s->c[i][2], s->p.nz));
                if (labels[nb] != -2) continue;
                labels[nb] = (int)start;
                queue[tail++] = nb;
            }
        }
    }
    free(queue);
    return count;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
