/*
 * lbref.h -- plain FP64 CPU oracle of one lattice time step of the
 * self-diffusiophoretic lattice Boltzmann model (free-energy binary fluid with
 * a solute, Sec. "Computational model", Eqs. free_energy, chem_potentials,
 * diffusion_reaction; particles by bounce-back on links with phoretic slip,
 * Janus activity and wetting, Sec. "Particles").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * definition the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It shares
 * no code, header or table with the CUDA library.
 *
 * Conventions (chosen to match the public data format of the library, which
 * is an interface and therefore has to agree):
 *   node index n = x + nx*(y + ny*z);  populations are [19][N];
 *   velocity arrays are [3][N];  all values are FP64.
 *   D3Q19 order: 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *   7..18 = (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
 *           (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 */
#ifndef LBREF_H
#define LBREF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ref_sim ref_sim;

typedef struct {
    int nx, ny, nz;
    int periodic[3];        /* 0 on an axis = halfway bounce-back walls */
    double tau, rho0;       /* BGK relaxation time, reference density    */
    double body_force[3];   /* uniform force density on the fluid        */
    double A, kappa, M_psi; /* Landau A (B = -A), gradient kappa, mobility */
    double C, M_phi, E, phi_b, k_d; /* solute stiffness, mobility, solubility,
                                       background, degradation rate      */
    int thermo_force;       /* 1: force -psi grad mu_psi - phi grad mu_phi */
    int scalar_scheme;      /* psi, phi transport: 0 finite differences on D3Q19
                               links; 1 lattice Boltzmann, D3Q7 distributions  */
} ref_params;

typedef struct {
    double pos[3], m_hat[3];
    double R, rho_p, alpha, mu_plus, mu_minus;
    double H;               /* surface field (already mapped from theta_c) */
    double vel[3], omega[3];
    double ext_force[3], ext_torque[3];
    int fixed;              /* 1: velocity and spin held at vel/omega      */
} ref_particle_desc;

typedef struct {
    double pos[3], vel[3], omega[3], m_hat[3], force[3], torque[3];
} ref_particle_state;

ref_sim* ref_create(const ref_params* p);
void     ref_destroy(ref_sim* s);
/* rho [N], u [3][N], psi [N], phi [N]; NULL keeps the current field.
 * Populations are reset to the equilibrium of (rho, u). */
int  ref_set_fields(ref_sim* s, const double* rho, const double* u,
                    const double* psi, const double* phi);
int  ref_add_particle(ref_sim* s, const ref_particle_desc* d);
int  ref_step(ref_sim* s, int nsteps);
int  ref_read_fields(const ref_sim* s, double* rho, double* u, double* psi,
                     double* phi);
int  ref_read_mu(ref_sim* s, double* mu_psi, double* mu_phi); /* of the current fields */
int  ref_read_populations(const ref_sim* s, double* f);
int  ref_read_mask(const ref_sim* s, unsigned char* mask);
int  ref_read_particles(const ref_sim* s, ref_particle_state* out, int cap);
int  ref_conservation(const ref_sim* s, double sums[3]);
int  ref_error(const ref_sim* s);
long ref_fluid_count(const ref_sim* s);
/* threads of the node loops (0: all cores); returns the count in use, 1
 * without OpenMP.  Results are bit-identical for any count. */
int  ref_set_threads(int n);
/* contact angle (degrees) -> h = H / sqrt(kappa A) by bisection */
double ref_wetting_h(double theta_deg);

#ifdef __cplusplus
}
#endif
#endif
