/*
 * lbdp_batch.h -- many independent boxes of the lattice update in lbdp.h,
 * advanced together on one GPU, and a continuous-batching request loop on
 * top of them.
 *
 * The paper runs one simulation at a time and has no counterpart of this
 * layer; every box computes exactly the step lbdp.h documents (Sec.
 * "Computational model", Sec. "Particles"), and a box gives identical bits
 * alone (lb_step) and inside a batch (lbb_run), in every precision mode.
 *
 * Conventions are those of lbdp.h: LB_OK or a negative LB_ERR_* status, no
 * exceptions across the ABI, FP64 host data, the caller owns host arrays.
 * A batch and its member boxes share one stream; none of these objects is
 * thread-safe.
 */
#ifndef LBDP_BATCH_H
#define LBDP_BATCH_H

#include <stddef.h>

#include "lbdp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------
 * Arena bookkeeping (host only, no device calls).  A batch places its boxes
 * in one device allocation managed by exactly this first-fit allocator with
 * coalescing: offsets are multiples of 256 bytes, a request of b bytes takes
 * b rounded up to 256.  Exposed so that admission decisions ("does a box of
 * this size fit now?") can be planned and tested without a GPU.
 * ------------------------------------------------------------------------ */
typedef struct lb_arena lb_arena;

/* capacity > 0 bytes (rounded down to 256).  LB_ERR_PARAM, LB_ERR_NOMEM. */
int lb_arena_create(size_t capacity, lb_arena** out);
/* First fit: the lowest free offset with room.  LB_ERR_NOMEM when no free
 * range holds the request (nothing changes); LB_ERR_PARAM for bytes == 0. */
int lb_arena_alloc(lb_arena* a, size_t bytes, size_t* offset);
/* Free the range that starts at offset; LB_ERR_PARAM if no range starts
 * there.  Adjacent free ranges merge. */
int lb_arena_free(lb_arena* a, size_t offset);
/* used: bytes held; largest_free: longest free range; free_ranges: count. */
int lb_arena_stats(const lb_arena* a, size_t* used, size_t* largest_free, int* free_ranges);
void lb_arena_destroy(lb_arena* a);

/* ------------------------------------------------------------------------
 * Batches
 * ------------------------------------------------------------------------ */
typedef struct lbb_batch lbb_batch;

typedef struct {
    int precision;       /* lb_precision of every member box                      */
    size_t arena_bytes;  /* device memory for member boxes, one cudaMalloc;
                            0 = three quarters of the free device memory          */
    int graph_steps;     /* steps captured per CUDA graph (>= 1); 0 = 16          */
    void* cuda_stream;   /* NULL = a stream the batch creates                     */
} lbb_params;

/* LB_ERR_PARAM (precision, negative graph_steps), LB_ERR_NOMEM, LB_ERR_CUDA. */
int lbb_create(const lbb_params* p, lbb_batch** out);
/* Destroys every member box, then the batch. */
void lbb_destroy(lbb_batch* b);

/* Arena bytes one box with these parameters takes (its region, rounded up
 * to 256).  LB_ERR_PARAM as lbb_add_box. */
int lbb_box_bytes(const lbb_batch* b, const lb_params* p, size_t* bytes);
int lbb_memory(const lbb_batch* b, size_t* capacity, size_t* used, size_t* largest_free);

/* Create a member box in the batch's arena, at rest as lb_create leaves it.
 * p->precision must equal the batch's; p->cuda_stream is ignored (members use
 * the batch stream); nx, ny <= 255 and nx*ny*nz < 2^24 (LB_ERR_PARAM).
 * LB_ERR_NOMEM when the arena has no room (the batch is unchanged).  The
 * handle works with every lb_* call; lb_destroy removes it from the batch and
 * returns its memory.  A new box has 0 steps to run. */
int lbb_add_box(lbb_batch* b, const lb_params* p, lb_handle** out);
int lbb_num_boxes(const lbb_batch* b);

/* Steps a member box still has to run (>= 0).  lbb_run advances a box only
 * while this is positive and counts it down. */
int lbb_set_steps(lbb_batch* b, lb_handle* h, long long nsteps);
int lbb_get_steps(const lbb_batch* b, const lb_handle* h, long long* left);

/* Run nsteps batch steps: in each, every box with steps left advances one
 * time step.  Full chunks of graph_steps run as one captured CUDA graph (one
 * graph launch), the rest as plain launches.  Queued on the batch stream;
 * returns without waiting.  launches (optional) receives the number of kernel
 * launches the call queued (graph nodes included). */
int lbb_run(lbb_batch* b, int nsteps, long long* launches);

/* Autotuning.  The two bulk kernels of a batched step -- the fused one
 * (chemical potentials, stress, force, collide-stream) and the transport --
 * march along z through 32 x 8 column tiles of every box; a block takes one z
 * chunk of a box.  The chunk length is the tuned shape: lbb_tune times each
 * candidate of each kernel over reps launches on the current boxes and keeps
 * the fastest.  The kernels only rewrite their own outputs (the stored
 * velocity is saved and restored), so tuning leaves the state unchanged.
 * cfg_out[LBB_KERNEL_CLASSES] (optional): the chosen candidate per kernel
 * (0 fused, 1 transport); ms_out (optional): its time per launch.  Results do
 * not depend on the configuration. */
#define LBB_KERNEL_CLASSES 2
int lbb_tune(lbb_batch* b, int reps, int cfg_out[LBB_KERNEL_CLASSES], double ms_out[LBB_KERNEL_CLASSES]);
/* Set the candidates directly (cfg[k] in [0, lbb_num_configs())). */
int lbb_set_config(lbb_batch* b, const int cfg[LBB_KERNEL_CLASSES]);
int lbb_num_configs(void);
/* Candidate k: threads per block and planes per block (the z chunk each
 * thread of the block marches through). */
int lbb_config_shape(int k, int* threads, int* planes);

/* Wait for the batch stream; report a device error of any member box. */
int lbb_sync(lbb_batch* b);

/* ------------------------------------------------------------------------
 * Continuous batching: requests arrive, are admitted into a batch as arena
 * memory frees up, run alongside whatever is already resident, and leave
 * with their results when their step count is reached.
 * ------------------------------------------------------------------------ */
typedef struct lbs_server lbs_server;

typedef struct {
    int precision;       /* of every request                                       */
    size_t arena_bytes;  /* as lbb_params                                          */
    int chunk_steps;     /* steps per lbs_pump round (>= 1); 0 = 64                */
    int max_boxes;       /* resident boxes at most; 0 = no limit                   */
    void* cuda_stream;
} lbs_params;

typedef struct {
    lb_params box;                   /* precision must match the server's           */
    int n_particles;                 /* 0..4                                        */
    lb_particle_desc particles[4];
    const double* psi;               /* initial fields [N] (host), NULL = 0; copied */
    const double* phi;               /*   at submission                             */
    long long steps;                 /* > 0                                         */
    double arrival;                  /* caller's clock (s) when the request arrived */
    double* out_psi;                 /* [N] host buffers for the final psi, phi      */
    double* out_phi;                 /*   (NULL = not returned); must stay valid    */
} lbs_request;                       /*   until the result is polled                */

typedef struct {
    long long id;
    int status;                      /* LB_OK or the box's error                    */
    double arrival, admitted, done;  /* caller's clock (s), see lbs_pump            */
    int n_particles;
    lb_particle_state particles[4];
    double sums[3];                  /* FP64 totals of rho, psi, phi at the end     */
} lbs_result;

int lbs_create(const lbs_params* p, lbs_server** out);
void lbs_destroy(lbs_server* s);
/* Queue a request (copied, initial fields included); *id receives its id.
 * LB_ERR_PARAM for invalid parameters or a box that can never fit. */
int lbs_submit(lbs_server* s, const lbs_request* r, long long* id);
/* One round: admit queued requests in arrival order while memory and slots
 * allow (a request that does not fit does not block smaller ones behind it),
 * run batch steps until the first resident box finishes, at most
 * chunk_steps, then retire the boxes that finished: copy out their results
 * and free their memory.  now is the caller's clock at the call; admitted and
 * done times are now plus the host time the round has taken until that
 * point.  *active and *queued (optional) receive the resident and waiting
 * request counts after the round. */
int lbs_pump(lbs_server* s, double now, int* active, int* queued);
/* Cancel request id between pumps: a queued request leaves the queue, a
 * resident one leaves the batch and frees its memory at once; either way its
 * result (status LB_ERR_CANCELLED, done = now, nothing written to its output
 * buffers) is posted for lbs_poll.  LB_ERR_PARAM for an id that is neither
 * queued nor resident (unknown, or already finished). */
int lbs_cancel(lbs_server* s, long long id, double now);
/* Finished results, oldest first; *n receives how many were written. */
int lbs_poll(lbs_server* s, lbs_result* out, int cap, int* n);
/* The batch the server runs (for tuning and diagnostics). */
lbb_batch* lbs_batch(lbs_server* s);

#ifdef __cplusplus
}
#endif

#endif /* LBDP_BATCH_H */
