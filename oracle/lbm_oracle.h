/*
 * FP64 CPU oracle of the thermal pseudopotential MRT lattice Boltzmann step of
 * Huang, Wang, He & Huang, "An efficient thermal lattice Boltzmann method for
 * simulating three-dimensional liquid-vapor phase change" (arXiv 2206.00946).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library. It shares no
 * code, header, table or helper with the CUDA library under
 * paper_2206_00946_gb300/; it follows the paper's equations literally (dense
 * matrix products M^-1 Lambda M, per-cell loops, no fusion) so that a reader can
 * check it against the paper by eye.
 *
 * Layout: cell index c = x + nx*(y + ny*z); populations f[i*N + c] (i = 0..18)
 * and g[i*N + c] (i = 0..6); all doubles.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NONFINITE = -3, ORC_ERR_PSI_DOMAIN = -4 };
enum { ORC_PERIODIC = 0, ORC_WALL = 1, ORC_OPEN = 2 };

typedef struct {
  int nx, ny, nz;
  double a, b, R, omega, G;          /* Peng-Robinson EOS (Sec. 4) and interaction strength (Eq. 6) */
  double s_e, s_v, s_q, s_pi;        /* D3Q19 relaxation rates in Lambda-hat (Eq. 10) */
  double cv, wbar;                   /* specific heat; D3Q7 rest-weight parameter (Eq. 14) */
  double lambda_l, lambda_v;         /* thermal conductivity of liquid / vapor */
  double rho_l, rho_v;               /* coexistence densities used to interpolate lambda */
  int vartheta;                      /* correction-term switch of Eq. 13 (0 or 1; 1 needs the T history) */
  int meq_printed;                   /* 1: rows 16-18 of m^eq exactly as printed in Eq. 9 */
  int wall_ueq_zero;                 /* 1: u^eq := 0 at bounce-back wall nodes (Sec. 3.1) */
  int eos_kind;                      /* 0: Peng-Robinson; 1: isothermal ideal gas p = c0*rho */
  double eos_c0;                     /* c0 of eos_kind 1 */
  int face_kind[6];                  /* faces -x,+x,-y,+y,-z,+z: ORC_PERIODIC/WALL/OPEN */
  double face_T[6];                  /* Dirichlet temperature of each non-periodic face */
  double face_rho[6];                /* prescribed density of an open (constant-pressure) face */
  double face_theta_deg[6];          /* contact angle of a wall face (Eq. 36) */
  int face_T_fixed[6];               /* 1: the node layer of face f holds the Dirichlet temperature
                                        face_T[f] even where the face is periodic for the flow
                                        (the droplet of Sec. 4.2: periodic velocity field,
                                        temperature fixed at the boundaries) */
} orc_params;

/* Optional per-cell fields at time t written by orc_step / orc_macros (NULL = skip). */
typedef struct {
  double *rho, *T, *psi, *p, *dpdT;  /* N each */
  double *ux, *uy, *uz;              /* real velocity, Eq. 5 (0 at wall nodes) */
  double *Fx, *Fy, *Fz;              /* interaction force, Eq. 6 */
} orc_fields;

/* thermodynamics (Sec. 4, Eqs. 37-38) */
double orc_Tc(const orc_params* P);
double orc_p_eos(const orc_params* P, double rho, double T);
double orc_dpdT(const orc_params* P, double rho, double T);
double orc_dpdrho(const orc_params* P, double rho, double T);
int orc_maxwell(const orc_params* P, double T, double* rho_v, double* rho_l, double* p_sat);

/* tables */
void orc_tables(int* c19, double* w19, int* c7, double* Mhat, double* Mhat_inv, double* M7, double* M7_inv);

/* per-cell pieces, exposed for the pins */
void orc_feq19(double rho, const double u[3], double feq[19]);
void orc_meq19(const orc_params* P, double rho, const double u[3], double meq[19]);
void orc_collide19(const orc_params* P, const double f[19], double rho, const double ueq[3],
                   const double F[3], double fstar[19]);
/* d2T: d^2T/dt^2 at the cell, entering through S_i of Eq. 16 when vartheta = 1 */
void orc_collide7(const orc_params* P, const double g[7], double rho, double T, const double u[3],
                  double divu, double dpdT, double d2T, double gstar[7]);
void orc_zouhe(const orc_params* P, int face, const double F[3], double f[19]);

/* whole-lattice operations.  Tface[f] (may be NULL) holds a per-node Dirichlet
 * temperature for face f, indexed by its two tangential coordinates (lower axis
 * fastest); NULL entries fall back to face_T[f]. */
int orc_check(const orc_params* P);
int orc_macros(const orc_params* P, const double* f, const double* g, orc_fields* out);
int orc_step(const orc_params* P, const double* const* Tface, const double* f, const double* g,
             double* f_out, double* g_out, orc_fields* diag);
int orc_run(const orc_params* P, const double* const* Tface, double* f, double* g, int nsteps);
/* vartheta = 1 (or 0): Th (2N) holds T at t-1 and t-2, and d^2T/dt^2 at t is the backward
 * second difference T(t) - 2 T(t-1) + T(t-2); Th_out (2N) receives T at t and t-1.
 * orc_step and orc_run take vartheta = 0 only.  The sign, size and leading-order effect of
 * S_i are pinned; the difference scheme is a reading (the paper names none): parity
 * unpinned for the scheme itself. */
int orc_step_hist(const orc_params* P, const double* const* Tface, const double* f, const double* g,
                  const double* Th, double* f_out, double* g_out, double* Th_out);
int orc_run_hist(const orc_params* P, const double* const* Tface, double* f, double* g, double* Th, int nsteps);
int orc_stream_map19(const orc_params* P, int* dst);
int orc_stream_map7(const orc_params* P, int* src);
int orc_node_class(const orc_params* P, unsigned char* cls);
void orc_init_state(const orc_params* P, const double* rho0, const double* T0, double* f, double* g);
/* threads of the per-cell loops (OpenMP build): n > 0 sets; returns the count in effect */
int orc_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
