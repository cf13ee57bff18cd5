/*
 * fre_oracle.h -- plain FP64 CPU oracle of the two-lattice free energy LBM
 * (Simonis et al., arXiv:2212.01617, Sec. 2.2 "Free energy lattice Boltzmann
 * method", Sec. 2.3 "Implementation", Algorithm 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists to check the CUDA path; it
 * is called by the tests, by __graft_entry__.smoke() and by the CPU-baseline
 * leg of bench.py, never by the product path.  It shares no code, header,
 * table or constant with the CUDA library (paper_2212_01617_gb300/csrc).
 *
 * Conventions (identical to the public C ABI in include/fre.h because they
 * are an interface, written out independently here):
 *   - node index n = (z*ny + y)*nx + x, x fastest;
 *   - populations are exchanged as FP64 arrays [q][n] in the canonical
 *     direction order listed in fre_oracle.c;
 *   - the state after k steps is the PRE-collision populations f(x,k), g(x,k)
 *     of the lattice Boltzmann equations (Eq. LBE, Eq. LBEg).
 */
#ifndef FRE_ORACLE_H
#define FRE_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1 };
enum { ORC_SHEAR = 0, ORC_FOUR_ROLLER = 1, ORC_PERIODIC = 2 };

typedef struct {
    int lattice;      /* ORC_D2Q9 or ORC_D3Q19 */
    int device;       /* ORC_SHEAR, ORC_FOUR_ROLLER or ORC_PERIODIC */
    int nx, ny, nz;   /* nz = 1 for D2Q9 */
    double tau_f;     /* relaxation time of f (Eq. bgk), > 0.5 */
    double tau_g;     /* relaxation time of g (Eq. LBEg), > 0.5 */
    double A;         /* bulk free-energy coefficient */
    double kappa;     /* gradient free-energy coefficient */
    double Gamma;     /* mobility parameter Gamma_phi (Eq. geq) */
    double u_wall;    /* shear: walls at -u_wall (bottom) / +u_wall (top);
                         four-roller: roller surface speed */
    double rho0;      /* reference density, also the wall density */
    int model;        /* 0: reduced functional (A, kappa; force -phi grad mu);
                         1: the full functional of Eq. functional (kappa1,
                         kappa2, alpha; force -rho grad mu_rho - phi grad mu_phi) */
    double kappa1, kappa2, alpha;
    int interp;       /* four-roller: 1 = interpolated bounce-back at the
                         roller surfaces (link fraction q from the circles),
                         0 = half-way bounce-back on the staircase */
} orc_params;

typedef struct {
    double mass, phi_sum, volume;
    double drop_weight, drop_count;
    double centroid[3];
    double I[6];      /* xx yy zz xy xz yz, central, normalised by drop_weight */
    double D, theta_deg;
    double p_centre, p_far, dp;
    double max_u;
    long long step;
    int status;       /* 0 ok, 1 non-finite value, 2 |u| > 0.3 */
} orc_obs;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_params *p);
void orc_destroy(orc_state *s);
int orc_q(const orc_state *s);
long long orc_nodes(const orc_state *s);
int orc_is_solid(const orc_state *s, int x, int y, int z);

int orc_init_droplet(orc_state *s, double cx, double cy, double cz, double R);
int orc_init_fields(orc_state *s, const double *rho, const double *ux,
                    const double *uy, const double *uz, const double *phi);
int orc_load_populations(orc_state *s, const double *f, const double *g);
int orc_store_populations(const orc_state *s, double *f, double *g);
int orc_step(orc_state *s, int nsteps);
int orc_fields(orc_state *s, double *rho, double *ux, double *uy, double *uz,
               double *phi, double *mu);
int orc_observables(orc_state *s, orc_obs *out);

/* Consistent initial populations (Sec. 2.3, Mei et al.): `iterations`
 * collide-and-stream passes of f with the velocity and force of the current
 * state held, rho free; g set to g_eq.  See fre_oracle.c. */
int orc_init_consistent(orc_state *s, int iterations);

/* Components of the phase phi > 0 (fluid nodes; phi given per node, n
 * values): labels[n] = -1 outside, else the smallest node index of the
 * component; returns the number of components.  See fre_oracle.c. */
int orc_label_phase(const orc_state *s, const double *phi, int *labels);

/* single-node building blocks, exposed so the tests can pin them */
int orc_lattice_info(int lattice, int *q, int *c /* q*3 */, double *w /* q */);
void orc_feq(int lattice, double rho, const double u[3], double *out);
void orc_geq(int lattice, double phi, double mu, double Gamma,
             const double u[3], double *out);
void orc_guo(int lattice, double tau, const double u[3], const double F[3],
             double *out);

int orc_num_threads(void);
void orc_set_num_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
