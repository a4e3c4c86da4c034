/*
 * mcg_oracle.h -- plain FP64 CPU oracle for the Feynman-Kac gravity walk.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  The product path
 * (the CUDA library and its Python binding) never calls it, links it or
 * includes this header; the two implementations share no code.
 *
 * What it computes (paper: Donzelli, Bihlo, Kischinhevsky, Farquharson,
 * "Massively parallel stochastic solution of the geophysical gravity
 * problem", arXiv:1709.07469):
 *   - the Feynman-Kac representation of the Dirichlet-Poisson problem
 *     (Sec. 2.1, Eq. 2-3 and its gravity form Eq. 5), restated for
 *     Delta Phi = 4 pi G rho with a standard Brownian motion:
 *       Phi(x0) = E[ g(W_tau) ] - 1/2 E[ int_0^tau 4 pi G rho(W_t) dt ];
 *   - the walk of Sec. 2.3 (Euler-Maruyama step, trapezoid rule for the
 *     source integral, exit check) with the last segment clipped to the box;
 *   - the Monte Carlo average of Eq. 7, plus the sample variance and the
 *     standard error;
 *   - g_z = dPhi/dz by the centred difference of Sec. 4.2 (experiment 3),
 *     with common random numbers.
 * Parity status of every function is listed in its comment.
 */
#ifndef MCG_ORACLE_H
#define MCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_RHO_NONE = 0, ORC_RHO_SPHERE = 1, ORC_RHO_PRISM = 2, ORC_RHO_VOXEL = 3 };
enum { ORC_G_ZERO = 0, ORC_G_SPHERE = 1, ORC_G_PRISM = 2, ORC_G_TABLE = 3, ORC_G_POLY = 4 };
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_STEP_CAP = 4 };

enum { ORC_DOMAIN_BOX = 0, ORC_DOMAIN_BALL = 1 };

typedef struct {
    double lo[3], hi[3];           /* box domain Omega = (lo, hi) open      */
    int    domain_kind;            /* box, or the ball |x - bc| < R         */
    double bc[3], R;
    int    rho_kind;
    double G;                      /* gravitational constant                */
    double rho0;                   /* sphere / prism density                */
    double center[3], radius;      /* sphere                                */
    double plo[3], phi[3];         /* prism [plo, phi) half-open            */
    const float* grid;             /* voxel grid, x fastest, nx*ny*nz       */
    int64_t n[3];
    double origin[3], spacing[3];
    int    g_kind;
    const float* faces;            /* 6 faces (-x,+x,-y,+y,-z,+z), nv*nu    */
    int32_t nu, nv;
    double poly[11];               /* 1,x,y,z,x2,y2,z2,xy,yz,zx,xyz          */
    double dt, sigma, h;           /* time step, diffusion scale, FD step   */
    uint64_t seed;
    int    clip;                   /* 1: clip last segment to the box       */
    int    crn;                    /* 1: walk x0, x0+h ez, x0-h ez together */
    int    ubits;                  /* 32: u=(w+.5)2^-32 ; 23: u=((w>>9)+.5)2^-23 */
    int64_t max_steps;             /* cap on RNG-steps per path             */
    int    bridge;                 /* 1: Brownian-bridge exit test on inside steps */
} orc_problem;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Pinned against the
 * cuRAND host generator (library, black box). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void orc_philox_fill(const uint32_t* ctrs, const uint32_t* keys, int64_t n, uint32_t* out);

/* Twelve standard normals of step block b of path (s, p): three Philox
 * calls with counters (3b+i, p, s, tag), i = 0,1,2, six Box-Muller pairs. */
void orc_normals_block(uint64_t seed, uint32_t s, uint32_t p, uint32_t b,
                       uint32_t tag, int ubits, double z[12]);
void orc_normals_fill(uint64_t seed, uint32_t s, uint32_t p, uint32_t b0,
                      int64_t nblocks, uint32_t tag, int ubits, double* z);

/* Density and boundary data. */
double orc_rho(const orc_problem* P, const double x[3]);
double orc_g(const orc_problem* P, const double x[3]);

/* Closed forms (pinned by far-field, additivity, Laplacian and FD tests). */
double orc_sphere_phi(double G, double rho0, const double c[3], double a, const double x[3]);
double orc_sphere_gz(double G, double rho0, const double c[3], double a, const double x[3]);
double orc_prism_phi(double G, double rho0, const double lo[3], const double hi[3], const double x[3]);
double orc_prism_gz(double G, double rho0, const double lo[3], const double hi[3], const double x[3]);

/* One path.  u[c] = per-copy estimate, steps[c] = EM steps taken by copy c,
 * xexit[3c..3c+2] = exit point of copy c.  Returns ORC_OK or an error. */
int orc_walk_path(const orc_problem* P, const double x0[3], uint32_t s, uint32_t p,
                  double u[3], int64_t steps[3], double xexit[9]);

/* Station solve over paths p0 .. p0+N-1 of every station.  Per-path arrays
 * (S*N, station-major) are optional.  Statistics are the two-pass sample
 * mean and variance, summed with Neumaier compensation in path order. */
int orc_solve(const orc_problem* P, const double* stations, int64_t S,
              int64_t p0, int64_t N, int nthreads,
              double* u, double* gz, double* se_u, double* se_gz,
              int64_t* path_steps,
              double* pp_u, double* pp_d, int64_t* pp_steps, int64_t* pp_copy_steps);

/* Setup of the heterogeneous model: Gaussian random field density and
 * boundary tables by direct prism summation. */
void orc_grf_density(uint64_t seed, int64_t nx, int64_t ny, int64_t nz,
                     double sigma_vox, double amp, float* grid_out, double* z_out);
int  orc_table_nodes(const orc_problem* P, const int64_t* face, const int64_t* iu,
                     const int64_t* iv, int64_t n, int nthreads, double* out);
/* Potential and dPhi/dz of the voxel model at arbitrary points (direct sum
 * of the prism closed forms over all voxels). */
int  orc_voxel_field(const orc_problem* P, const double* x, int64_t n, int nthreads,
                     double* phi, double* gz);

#ifdef __cplusplus
}
#endif
#endif
