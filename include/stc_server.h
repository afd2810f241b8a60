/*
 * stc_server.h -- serving many smoke-control problems on one GPU.
 *
 * The paper solves one problem at a time.  This layer keeps several problems
 * resident and solving at once: requests of different grid sizes, timestep
 * counts and keyframe sets are admitted against a device-memory budget and
 * each admitted problem runs the ADMM loop of Alg. 3 (stc_solve) on its own
 * CUDA stream, with its own captured V-cycle graph, so the launches of all
 * resident problems interleave on the device.  A request is admitted as soon
 * as a worker and enough of the budget are free (first fit over the queue in
 * arrival order; a request passed over max_bypass times blocks later ones
 * until it fits), and its memory returns to the budget the moment its solve
 * ends.  The admission size of a request is stc_problem_bytes (the exact
 * device bytes of the problem), the analogue for this library of the memory
 * bound M ~ 8 n^d (1 + d) N of Sec. 5.
 *
 * Two modes.  Mode 0 (worker threads): each admitted problem runs stc_solve
 * on its own stream and the launches of all resident problems interleave.
 * Mode 1 (stepped): the caller drives stc_server_step.  A step admits what
 * fits, starts background jobs (one host thread and the problem's own stream
 * each) for the set-up of admitted problems, the AO head (Alg. 1) of problems
 * whose ADMM iteration begins and the KKT/update tail of problems whose NSO
 * solve ended, then runs ONE batched CUDA graph launch holding the next NSO
 * V-cycle of every idle problem (stc_batch_nso_cycle: the problems' captured
 * V-cycle graphs as concurrent child nodes; the instantiated graph is reused
 * while that set stays the same), and retires finished problems, returning
 * their memory at once -- continuous batching at V-cycle granularity, with
 * heads and tails overlapping the batched V-cycles on the device.  The
 * batched launches run on stc_server_params.stream.
 *
 * Threading: every stc_server_* call is safe from any host thread (stepped
 * steps are serialised).  Results are copied to host memory owned by the
 * server until stc_server_release.
 *
 * Errors: as in stc.h; stc_last_error() describes the last failing call of
 * the calling thread.  A request whose solve fails ends in state
 * STC_TICKET_FAILED with its status and message in stc_ticket_info; the
 * server and the other requests carry on.
 */
#ifndef STC_SERVER_H
#define STC_SERVER_H

#include "stc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stc_server stc_server; /* opaque */

typedef struct {
  size_t budget_bytes; /* device bytes the resident problems may hold together        */
  int workers;         /* problems solved at once (host threads, one stream each); >= 1 */
  int backend;         /* 0 = the GPU library; 1 = simulated solves on the host only
                          (no CUDA call: sleeps sim_seconds and ends with sim_status;
                          for testing the scheduler without a GPU)                      */
  int device;          /* CUDA device of the GPU backend                                */
  int max_bypass;      /* times a queued request may be passed over by later ones (8)  */
  int mode;            /* 0 (default): worker threads; 1: stepped (stc_server_step)    */
  void* stream;        /* mode 1: CUDA stream of the batched launches (NULL = legacy
                          default stream)                                             */
  int max_resident;    /* mode 1: problems solving at once (16)                         */
  double kkt_rel_tol;  /* mode 1: stopping tolerance of problems submitted with
                          stc_server_submit_problem (1e-4)                            */
  int max_admm;        /* mode 1: their ADMM iteration cap (50)                         */
} stc_server_params;

typedef struct {
  const stc_params* params;  /* copied at submit                                        */
  const double* rho0;        /* nx*ny cells, copied                                     */
  const double* v0;          /* faces or NULL (= 0), copied                             */
  int nkeys;                 /* keyframes (steps 1..N), copied                          */
  const int* key_steps;
  const double* key_rho;     /* nkeys x nx*ny                                           */
  const double* key_c;       /* NULL = 1                                                */
  double kkt_rel_tol;        /* stc_solve's tolerance                                  */
  int max_admm;              /* stc_solve's iteration cap                              */
  double sim_seconds;        /* simulated backend: duration of the solve               */
  int sim_status;            /* simulated backend: status the solve ends with          */
} stc_request;

typedef enum {
  STC_TICKET_QUEUED = 0,
  STC_TICKET_RUNNING = 1,
  STC_TICKET_DONE = 2,       /* stc_solve returned STC_OK or STC_ERR_NOT_CONVERGED      */
  STC_TICKET_FAILED = 3,     /* any other status                                       */
  STC_TICKET_CANCELLED = 4
} stc_ticket_state;

typedef struct {
  int state;                 /* stc_ticket_state                                       */
  int status;                /* stc_status of the solve (DONE / FAILED)                */
  size_t bytes;              /* admission size                                         */
  double t_submit, t_admit, t_done; /* seconds since stc_server_create (-1: not yet)   */
  stc_report report;         /* stc_solve's report (DONE / FAILED)                     */
  char error[160];           /* message of a failed solve                              */
} stc_ticket_info;

typedef struct {
  int queued, running, done, failed, cancelled;
  size_t bytes_in_use, peak_bytes;
} stc_server_stats;

void stc_server_default_params(stc_server_params* sp, size_t budget_bytes);
stc_status stc_server_create(const stc_server_params* sp, stc_server** out);
/* Queues a request.  STC_ERR_INVALID_ARG for malformed requests and
 * STC_ERR_OOM when the request alone exceeds the budget (never admissible). */
stc_status stc_server_submit(stc_server* s, const stc_request* rq, long long* ticket);
/* Mode 1: queues a problem the caller created (on any stream of the server's
 * device, with its keyframes set), solved with the server's kkt_rel_tol and
 * max_admm.  Its
 * admission size is stc_memory_bytes(problem) (already allocated: the budget
 * bounds how many problems solve at once).  The server does not destroy it;
 * the caller must not use it until the ticket is finished.  STC_ERR_INVALID_ARG
 * in mode 0, STC_ERR_OOM when it alone exceeds the budget. */
stc_status stc_server_submit_problem(stc_server* s, stc_problem* problem, long long* ticket);
/* Mode 1: one serving step (see above); *active (may be NULL) = problems
 * resident or queued after it.  Failures of single problems end their
 * tickets (FAILED) and the step carries on.  STC_ERR_INVALID_ARG in mode 0. */
stc_status stc_server_step(stc_server* s, int* active);
stc_status stc_server_poll(stc_server* s, long long ticket, stc_ticket_info* info);
/* Blocks until the ticket is DONE, FAILED or CANCELLED, or timeout_s elapses
 * (timeout_s < 0: no limit); info receives the state either way.  In mode 1
 * the waiting thread runs stc_server_step itself until then (or until no
 * problem is left). */
stc_status stc_server_wait(stc_server* s, long long ticket, double timeout_s, stc_ticket_info* info);
/* Cancels a queued request; a running one is not interrupted (STC_ERR_BUSY). */
stc_status stc_server_cancel(stc_server* s, long long ticket);
/* Forces u_i, i = 0..N-1 (N x faces, as stc_get_forces) of a DONE ticket. */
stc_status stc_server_get_forces(stc_server* s, long long ticket, double* u, size_t len);
/* Frees a finished ticket's record and result. */
stc_status stc_server_release(stc_server* s, long long ticket);
stc_status stc_server_stats_get(stc_server* s, stc_server_stats* out);
/* Cancels queued requests, waits for running ones, frees everything. */
stc_status stc_server_destroy(stc_server* s);

#ifdef __cplusplus
}
#endif

#endif
