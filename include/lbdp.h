/*
 * lbdp.h -- C ABI of the GB300 lattice Boltzmann library for self-diffusiophoretic
 * particles near liquid-liquid interfaces (arXiv 2202.01631).
 *
 * One simulation box lives on one GPU.  A time step is the coupled update of
 *   - the D3Q19 BGK solvent (Sec. "Computational model", nu = (tau - 1/2)/3),
 *   - the water/oil order parameter psi and the solute phi through their
 *     chemical potentials (Eqs. free_energy, chem_potentials,
 *     diffusion_reaction), with Janus production on the catalytic cap
 *     (Eq. activity) and the degradation sink k_d (phi - phi0(psi)),
 *   - spheres coupled by bounce-back on links with momentum-exchange force and
 *     torque, phoretic slip v_s = mu (1 - n n) . grad phi with Janus mobility
 *     (Eq. MuJ), wetting through the surface field H (Eq. fe_wetting and the
 *     contact-angle relation), and node covering/uncovering as they move
 *     (Sec. "Particles").
 *
 * Conventions shared by every entry point
 *   - Node index n = x + nx*(y + ny*z); scalar fields are [N] arrays, vectors
 *     [3][N] (component-major), populations [19][N] in the D3Q19 order
 *       0 rest; 1..6 +x,-x,+y,-y,+z,-z;
 *       7..18 (+1,+1,0),(-1,-1,0),(+1,-1,0),(-1,+1,0),(+1,0,+1),(-1,0,-1),
 *             (+1,0,-1),(-1,0,+1),(0,+1,+1),(0,-1,-1),(0,+1,-1),(0,-1,+1).
 *   - Host data crossing the ABI is FP64 in every precision mode.  The
 *     caller owns every host array; the library copies in and out and owns
 *     all device memory of a handle.
 *   - Nodes inside a particle read back as 0 in every field.
 *   - Every call returns LB_OK (0) or a negative LB_ERR_* status; no C++
 *     exception crosses the ABI.  A handle is not thread-safe.
 *   - Work is queued on the handle's stream (lb_params.cuda_stream, or a
 *     stream the library creates when it is NULL).  lb_step returns without
 *     waiting; the read and conservation calls synchronise the stream.
 *     Errors detected on the device (a particle leaving the allowed region,
 *     two particles meeting) are reported by the next synchronising call.
 */
#ifndef LBDP_H
#define LBDP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lb_handle lb_handle;

/* Storage and arithmetic precision of a box.
 *   LB_FP64        populations and fields FP64, FP64 arithmetic.
 *   LB_FP32        populations stored FP32 as f_i - w_i rho0, FP32 arithmetic.
 *   LB_FP16_SHIFT  populations stored FP16 as (f_i - w_i rho0)/w_i, FP32
 *                  fields and arithmetic.
 *   LB_BF16_SHIFT  as LB_FP16_SHIFT with BF16 storage.
 * Particle state, force/torque sums and conservation sums are FP64 always. */
enum {
    LB_FP64 = 0,
    LB_FP32 = 1,
    LB_FP16_SHIFT = 2,
    LB_BF16_SHIFT = 3
};

enum {
    LB_OK = 0,
    LB_ERR_PARAM = -1,     /* invalid argument or parameter set            */
    LB_ERR_NOMEM = -2,     /* device allocation failed                     */
    LB_ERR_NONFINITE = -3, /* a conserved total became NaN or Inf          */
    LB_ERR_OVERLAP = -4,   /* particles met, or a particle reached a wall  */
    LB_ERR_CUDA = -5,      /* a CUDA call failed                           */
    LB_ERR_TIMEOUT = -6,   /* reserved: a bounded device wait expired      */
    LB_ERR_STATE = -7,     /* call not valid in the handle's current state */
    LB_ERR_CANCELLED = -8  /* a served request was cancelled (lbs_cancel)  */
};

/* Box and model parameters (Sec. "Numerical details" gives the paper's
 * values: tau = 1 (nu = 1/6), rho0 = 1, A = C = 0.0625, kappa = 0.04). */
typedef struct {
    int nx, ny, nz;         /* lattice size, unit spacing                   */
    int periodic[3];        /* 1 periodic; 0 halfway bounce-back walls at
                               -1/2 and n-1/2 with neutral wetting          */
    int precision;          /* LB_FP64 ... LB_BF16_SHIFT                    */
    int thermo_force;       /* 1 (default model): fluid force g - div P,
                               P the pressure tensor of the free energy
                               (Eq. free_energy), in link form
                               -6 sum_i w_i [(P(x) + P(x+c_i))/2] . c_i with
                               P(x) standing in at solid and wall
                               neighbours; its continuum value is
                               -psi grad mu_psi - phi grad mu_phi, and each
                               boundary link hands a particle 6 w_i P(x).c_i;
                               0: psi and phi are passive scalars           */
    double tau, rho0;       /* BGK relaxation time (> 1/2), reference density */
    double body_force[3];   /* uniform force density g on the fluid         */
    double A, kappa, M_psi; /* Landau double well A psi^4/4 - A psi^2/2,
                               gradient coefficient, psi mobility           */
    double C, M_phi;        /* solute stiffness and mobility (D = C M_phi)  */
    double E, phi_b;        /* solubility: phi0(psi) = phi_b + E tanh psi   */
    double k_d;             /* degradation rate of the sink                 */
    void* cuda_stream;      /* cudaStream_t to queue work on, or NULL       */
    int scalar_scheme;      /* transport of psi and phi (Eq. diffusion_reaction):
                               0 conservative finite differences on the D3Q19
                               links (donor-cell advection);
                               1 lattice Boltzmann: D3Q7 distributions with
                               relaxation time 1 whose equilibrium carries the
                               chemical potential (mobility M = Gamma/2) and
                               moving-wall bounce-back at particles.  With
                               relaxation time 1 the post-collision
                               distributions are functions of the node's
                               fields, so none are stored.  Other values:
                               LB_ERR_PARAM                                */
} lb_params;

/* One sphere (Sec. "Particles").  pos must keep the sphere one node clear of
 * any wall and of other spheres.  m_hat need not be normalised.
 * theta_c_deg sets the contact angle through
 *   cos(theta_c) = [(1+h)^{3/2} - (1-h)^{3/2}]/2,  H = h sqrt(kappa A);
 * when theta_c_deg is NaN, H is taken as given.  The cap m.n <= 0 produces
 * solute at rate alpha per adjacent fluid node and per step, with mobility
 * mu_minus there and mu_plus on the other hemisphere (Eqs. activity, MuJ).
 * rho_p <= 0 means 1.  fixed != 0 holds vel/omega constant (the sphere still
 * moves at vel and turns at omega; the force it feels is reported).
 * ext_force/ext_torque are constant external loads. */
typedef struct {
    double pos[3], m_hat[3];
    double R, rho_p, alpha, mu_plus, mu_minus;
    double theta_c_deg, H;
    double vel[3], omega[3];
    double ext_force[3], ext_torque[3];
    int fixed;
} lb_particle_desc;

/* State after the last step; force/torque are the totals the particle felt
 * in that step (hydrodynamic, covering impulses and external). */
typedef struct {
    double pos[3], vel[3], omega[3], m_hat[3], force[3], torque[3];
} lb_particle_state;

/* Create a box: validates params (LB_ERR_PARAM), allocates the device state
 * (LB_ERR_NOMEM), and sets the fluid at rest with rho = rho0, psi = phi = 0.
 * On success *out receives the handle; on failure *out is NULL. */
int lb_create(const lb_params* params, lb_handle** out);

/* Release every device allocation of the handle.  NULL is ignored. */
void lb_destroy(lb_handle* h);

/* Set the fields from host arrays rho [N], u [3][N], psi [N], phi [N] (any may
 * be NULL to keep the current field) and reset the populations to the
 * second-order equilibrium of (rho, u) (Sec. "Numerical details": the system
 * starts from equilibrium).  Values at nodes inside particles are ignored.
 * A NaN or Inf in a given array (at any node) returns LB_ERR_NONFINITE and
 * leaves the box unchanged. */
int lb_set_fields(lb_handle* h, const double* rho, const double* u,
                  const double* psi, const double* phi);

/* Add a sphere (Sec. "Particles").  Nodes whose centre lies strictly inside
 * the sphere become solid and their fields are dropped.  Returns
 * LB_ERR_PARAM for a bad descriptor, LB_ERR_OVERLAP if it meets a wall or
 * another sphere.  *id_out (may be NULL) receives the particle index. */
int lb_add_particle(lb_handle* h, const lb_particle_desc* desc, int* id_out);

/* Queue nsteps time steps (nsteps >= 0) on the handle's stream and return
 * without waiting.  Each step: chemical potentials (Eq. chem_potentials);
 * force, streaming with bounce-back and BGK collision; psi/phi transport
 * (Eq. diffusion_reaction); particle update; covering/uncovering.  The
 * particle kernels run on a second stream of the library's that joins the
 * handle's stream before each step ends.  A box without particles runs whole
 * groups of 8 steps as one captured CUDA graph (captured on first use and
 * again after its parameters or launch grids change); while the caller is
 * itself capturing the handle's stream, and on the legacy default stream,
 * every step is launched plainly.  Results do not depend on the route. */
int lb_step(lb_handle* h, int nsteps);

/* Run nsteps steps like lb_step, but with every kernel on the handle's stream
 * in sequence and a CUDA event recorded between kernel classes; wait, and add
 * each class's time in milliseconds to ms[0..4]:
 *   0 the particle kernels before the bulk: pressure tensor and force at the
 *     fluid nodes next to particles, particle links and velocity update,
 *     collide-stream of the fluid nodes next to particles;
 *   1 chemical potentials, pressure tensor, force and collide-stream of all
 *     other fluid nodes (one fused kernel);
 *   2 psi/phi transport of the fluid nodes not next to particles (one kernel);
 *   3 psi/phi transport of the fluid nodes next to particles;
 *   4 covering/uncovering.
 * *launches (may be NULL) receives the number of kernels launched.  The
 * events add a little host overhead, so time throughput with lb_step; this
 * call is for the split. */
int lb_profile_step(lb_handle* h, int nsteps, double* ms, int* launches);

/* Autotuning.  The two bulk kernels (the fused chemical potentials, stress,
 * force and collide-stream, and the psi/phi transport) march along z through
 * 32 x 8 column tiles; a block takes one z chunk.  Short chunks recompute
 * more halo planes, long ones leave SMs idle, and the best length depends on
 * the box, so lb_tune times each kernel alone over reps launches for chunk
 * lengths from 4 to 64 planes (each rounded to equal chunks) and keeps the
 * fastest per kernel.  The kernels only rewrite the next step's buffers and
 * the stored velocity, which is saved and restored: the state is unchanged,
 * and the results of later steps do not depend on the chunk length (bit for
 * bit).  planes_out[2], ms_out[2] (optional): the chosen lengths and their
 * times per launch (0 fused, 1 transport).  Synchronises.  LB_ERR_PARAM for
 * reps < 1. */
int lb_tune(lb_handle* h, int reps, int planes_out[2], double ms_out[2]);
/* Set the chunk lengths directly; 0 restores the size heuristic (a chunk
 * count of about six waves of four blocks per SM, chunks of at least 6
 * planes); lengths above nz are clamped.  LB_ERR_PARAM for a negative one. */
int lb_set_planes(lb_handle* h, const int planes[2]);
/* The chunk lengths the next lb_step uses (after rounding to equal chunks). */
int lb_get_planes(const lb_handle* h, int planes[2]);

/* Number of kernels lb_step(h, nsteps) launches (for launch accounting). */
int lb_step_launches(const lb_handle* h, int nsteps);

/* Wait for queued work and report device-side errors. */
int lb_sync(lb_handle* h);

/* Copy the fields to host arrays (any may be NULL): rho = sum_i f_i,
 * u = velocity of the last collision (with the half-force term), psi, phi.
 * Synchronises. */
int lb_read_fields(lb_handle* h, double* rho, double* u, double* psi, double* phi);

/* Copy the chemical potentials mu_psi, mu_phi [N] of the current fields
 * (Eq. chem_potentials).  Synchronises. */
int lb_read_mu(lb_handle* h, double* mu_psi, double* mu_phi);

/* Copy the post-collision populations f_i [19][N] (FP64).  Synchronises. */
int lb_read_populations(lb_handle* h, double* f);

/* Copy the solid mask [N]: 0 fluid, k+1 inside particle k.  Synchronises. */
int lb_read_mask(lb_handle* h, unsigned char* mask);

/* Checkpoint and restart (no counterpart in the paper: a run can be stopped
 * and continued).  lb_state_bytes gives the size of a checkpoint of h.
 * lb_save_state copies the whole state after the last step into the host
 * buffer buf (bytes >= lb_state_bytes, else LB_ERR_PARAM): populations,
 * psi, phi and u in the box's storage precision, the solid mask and the
 * boundary flags, every particle record (position, velocity, spin,
 * orientation and the covering impulses it carries into the next step), the
 * pending uniform psi/phi correction, the fluid-node count and the error
 * word.  Synchronises.  lb_load_state restores such a checkpoint into a box
 * created with the same lattice size, axes, precision, transport scheme and
 * model parameters (LB_ERR_PARAM otherwise, nothing changed); its particles
 * are replaced by the checkpoint's.  A box of a batch cannot be restored into
 * (LB_ERR_STATE).  Stepping the restored box then gives the
 * same bits as stepping the saved one. */
int lb_state_bytes(const lb_handle* h, size_t* bytes);
int lb_save_state(lb_handle* h, void* buf, size_t bytes);
int lb_load_state(lb_handle* h, const void* buf, size_t bytes);

/* Copy up to cap particle states; *n_out (may be NULL) gets the count. */
int lb_read_particles(lb_handle* h, lb_particle_state* out, int cap, int* n_out);

/* FP64 totals over fluid nodes: sums[0] = sum rho, sums[1] = sum psi,
 * sums[2] = sum phi, reduced on the device in a fixed order.  Returns
 * LB_ERR_NONFINITE if any is NaN or Inf.  Synchronises. */
int lb_conservation(lb_handle* h, double sums[3]);

/* FP64 totals of caller-owned fields, computed without allocating device
 * memory.  The paper has no counterpart: this call exists for callers that
 * must not allocate -- a serving process whose device memory is planned and
 * owned by its own arena allocator, or a latency-critical loop that cannot
 * pay for the device-wide synchronisation cudaMalloc/cudaFree may imply.
 *
 * Inputs are device pointers in plain (unshifted) layout of the given
 * precision (LB_FP64 double or LB_FP32 float): populations f [19][N],
 * psi [N], phi [N], and mask [N] (u8, 0 = fluid; NULL counts every node).
 * sums (device, 3 doubles) receives sum rho = sum_i f_i, sum psi, sum phi
 * over the counted nodes, in the same fixed order on every call.  Work is
 * queued on stream (a cudaStream_t, NULL = legacy default stream) and the
 * call returns without waiting.
 *
 * Per-block partials live in one fixed 192 KiB array in the library's
 * device memory (3 doubles for each of 8192 blocks of 2048 nodes), which
 * every GPU that loads the library holds until the process exits.  Boxes of
 * more than 8192 * 2048 = 16,777,216 nodes (256^3) are rejected with
 * LB_ERR_PARAM before anything is queued.  The first call on each device
 * looks up that array's device address (cudaGetSymbolAddress), so make the
 * first call on a device before any stream capture.  All calls share the
 * array: each call overwrites every slot it reads, so nothing carries over,
 * but calls that overlap on the GPU (on different streams without ordering)
 * race on it.  No cudaMalloc, cudaFree or other allocating routine is
 * called.  Returns LB_OK, LB_ERR_PARAM or LB_ERR_CUDA. */
int lb_totals_noalloc(int precision, int nx, int ny, int nz, const void* f,
                      const void* psi, const void* phi, const unsigned char* mask,
                      double* sums, void* stream);

/* Device bytes lb_create would allocate for params (for admission control). */
int lb_device_bytes(const lb_params* params, size_t* bytes);

/* h = H / sqrt(kappa A) for a contact angle in degrees, by bisection of
 * cos(theta_c) = [(1+h)^{3/2} - (1-h)^{3/2}]/2 on [-1, 1]
 * (Sec. "Particles", contact-angle relation). */
double lb_wetting_h(double theta_c_deg);

/* Solubility parameter E for a ratio r = phi0(psi=+1)/phi0(psi=-1) of the
 * shifted minimum phi0 = phi_b + E tanh(psi) (Eq. free_energy):
 * E = phi_b (r - 1) / ((r + 1) tanh 1). */
double lb_solubility_E(double ratio, double phi_b);

/* Static message for a status code. */
const char* lb_error_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* LBDP_H */
