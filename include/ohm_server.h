/* ohm_server.h -- continuous-batching solve service on top of libohm (include/ohm.h).
 *
 * Not in the paper, which integrates one hierarchy: this is the deployment layer that serves
 * many independent ohmic-dissipation problems (Sec. 2.1: B^n, eta, dt -> B^{n+k}) on one GPU.
 * Requests are admitted as batch slots and device memory free up:
 *
 *   - requests with the same block structure and cell width form a class; a class is solved
 *     by batched hierarchies (ohm_cn_step_batch) of max_batch slots whose B, eta and
 *     multigrid scratch stay resident on the device between requests;
 *   - a request waits in a FIFO queue until a slot of its class is free; slots are refilled
 *     between the steps of a batch (continuous batching), so requests that arrive while
 *     others run join at the next step boundary;
 *   - up to n_workers batches run at once, each from its own host thread on its own stream,
 *     so their kernels overlap on the GPU;
 *   - a batch is created only if its device bytes (ohm_hierarchy_bytes plus B and eta) fit
 *     in hbm_budget_bytes beside the resident ones; idle batches are evicted (least recently
 *     used) to make room, otherwise the class waits.
 *
 * A request's result does not depend on which other requests share its batch or slot
 * (ohm_cn_step_batch gives each instance the same bits alone and in any batch).
 * All functions are thread safe. */
#ifndef OHM_SERVER_H
#define OHM_SERVER_H

#include <stdint.h>

#include "ohm.h"

#ifdef __cplusplus
extern "C" {
#endif

#define OHM_ERR_TIMEOUT (-6) /* ohm_server_wait: the request did not complete in time */

typedef struct ohm_server ohm_server;

typedef struct {
    int64_t hbm_budget_bytes;   /* device bytes the resident batches may hold (> 0)            */
    int32_t max_batch;          /* slots (instances) per batch, 1 .. 4096                      */
    int32_t n_workers;          /* batches in flight at once (host threads, streams), 1 .. 64  */
    int32_t precision;          /* OHM_FP64, OHM_MIXED or OHM_MIXED_FF                         */
    int32_t nu_pre, nu_post, n_coarse, max_outer;  /* multigrid schedule, as ohm_hier_desc   */
    double lambda;              /* theta parameter (0, 1]                                      */
    double tol;                 /* relative residual of every step (>= 0)                      */
    int32_t use_graphs;         /* 1: batches replay their inner iteration as a CUDA graph     */
    int32_t krylov;             /* OHM_MIXED(_FF): 0 = defect-correction inner solves, m in 1..11 =
                                   per-instance FGMRES(m) (see ohm_hier_desc)                  */
    double omega;               /* relaxation factor of the sweeps (see ohm_hier_desc); 0 = 1  */
    int32_t nu_coarse_pre, nu_coarse_post; /* sweeps on the coarser grids (see ohm_hier_desc)   */
} ohm_server_desc;

typedef struct {
    /* block structure of one instance, as in ohm_hier_desc (block_lijk copied by submit) */
    int32_t base_cells[3];
    double dx0;
    int32_t nlevels;
    int64_t nblocks;
    const int32_t *block_lijk;
    const double *B;            /* host [nblocks][3][8][8][8] initial field, copied by submit   */
    const double *eta;          /* host [nblocks][8][8][8] resistivity, copied by submit        */
    double dt;                  /* step, > 0                                                   */
    int32_t nsteps;             /* theta steps to take, >= 1                                   */
    double *B_out;              /* host [nblocks][3][8][8][8]: receives B after nsteps steps;
                                   must stay valid until ohm_server_wait returns for it        */
} ohm_request;

typedef struct {
    int32_t status;             /* OHM_OK, OHM_ERR_NOT_CONVERGED, OHM_ERR_NONFINITE, ...       */
    int32_t cycles;             /* V-cycles over all steps                                     */
    double rel_l2;              /* final ||R||/||S|| of the last step                          */
    double t_submit, t_start, t_done;  /* seconds on the server clock: queued, first step
                                          issued, result copied to B_out                      */
    int32_t slot;               /* batch slot that served the request                          */
} ohm_request_result;

typedef struct {
    int64_t requests_done;
    int64_t batches_created, batches_evicted;
    int64_t bytes_resident, bytes_resident_max;
    int64_t steps_run;          /* batched steps issued                                        */
    double mean_active_slots;   /* active slots per batched step                               */
    int64_t kernel_launches;    /* kernel launches issued by all batches so far                */
} ohm_server_stats;

/* Starts the worker threads on the calling thread's current CUDA device. */
int ohm_server_create(const ohm_server_desc *d, ohm_server **out);

/* Queues one request (copies B, eta and the block list); *id identifies it.  Returns
 * OHM_ERR_INVALID for a bad request or one whose batch alone exceeds the budget. */
int ohm_server_submit(ohm_server *s, const ohm_request *r, int64_t *id);

/* Waits up to timeout_s seconds (< 0: forever) for request id; on completion fills *res and
 * forgets the request.  OHM_ERR_TIMEOUT if it is still running, OHM_ERR_INVALID for an
 * unknown id. */
int ohm_server_wait(ohm_server *s, int64_t id, double timeout_s, ohm_request_result *res);

double ohm_server_clock(const ohm_server *s);
int ohm_server_get_stats(ohm_server *s, ohm_server_stats *st);

/* Finishes the queued and running requests, stops the workers, frees every batch. */
void ohm_server_destroy(ohm_server *s);

#ifdef __cplusplus
}
#endif
#endif /* OHM_SERVER_H */
