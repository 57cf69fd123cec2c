/*
 * sgtp.h -- C ABI of the B300 (sm_103a) SGTP best-response engine.
 *
 * SGTP (Li et al., "SGTP: Sampling-based Game-Theoretic Planning for
 * Real-Time Multi-Vehicle Autonomous Racing") plans by iterative best
 * response (Alg. 1).  Each best response samples K control sequences
 * around a nominal one (Sec. II, Algorithm Formulation), rolls them through
 * a kinematic bicycle model, scores them with the tracking cost (Eq. ctrack)
 * plus the game-aware cost (Eqs. game_cost, c_contest, c_long, c_block,
 * c_safety, allc), checks track boundaries and collisions (Eqs.
 * selection-boundary, selection-vehicle) and selects the lowest-cost
 * feasible sample (Eq. selection), falling back to the least violation.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All numeric arrays are float32, row-major and contiguous.  Arrays
 *    passed to the compute calls are DEVICE pointers owned by the caller;
 *    only sgtp_track_create* take HOST arrays.
 *  - States are [x, y, psi, v] (m, m, rad, m/s); controls are [a, delta]
 *    (m/s^2, rad) (Sec. II, Preliminaries).  Trajectories include tau = 0,
 *    so a trajectory of horizon T has T+1 states.
 *  - Lateral offset d > 0 is left of the raceline's direction of travel.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Compute calls only enqueue work: they return after launch-time
 *    validation, and device-side faults (a wait that timed out) are written
 *    to the caller's `status_dev` word, never by aborting the process.
 *  - A return of SGTP_E_INVALID means nothing was launched.  The text of the
 *    last error of the calling thread is returned by sgtp_last_error().
 *  - "No feasible sample" is not an error: it is reported per best response
 *    (any_feasible = 0) and the least-violation sample is returned
 *    (Sec. III-B, fallback).
 *  - Noise: sample k of a best response draws, at step tau, the Philox4x32-10
 *    block with key (seed lo32, seed hi32) and counter
 *    (k, (tau >> 1) | stream << 31, agent | round << 16, race); words 0,1
 *    serve even tau and words 2,3 odd tau.  A word w becomes the uniform
 *    u = ((w >> 9) + 0.5) * 2^-23 and a pair (u1, u2) the normals
 *    z_a = sqrt(-2 ln u1) cos(2 pi u2), z_delta = sqrt(-2 ln u1) sin(2 pi u2)
 *    (Box-Muller).  eps = (sigma_a z_a, sigma_delta z_delta).  stream is 0
 *    for the plain Gaussian sampler.
 *  - Workspace: calls that need device scratch take (workspace, bytes); the
 *    caller allocates it (any device allocation, 256-byte aligned) and may
 *    reuse it across calls on the same stream.  The library never allocates
 *    inside a compute call.
 */
#ifndef SGTP_H
#define SGTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sgtp_status;
enum {
    SGTP_OK = 0,
    SGTP_E_INVALID = 1,   /* bad argument; nothing launched                         */
    SGTP_E_CUDA = 2,      /* a CUDA runtime call failed (text in sgtp_last_error)   */
    SGTP_E_NOMEM = 3,     /* setup-time allocation failed                           */
    SGTP_E_TIMEOUT = 4,   /* a device-side wait ran past its limit and gave up      */
    SGTP_E_DEVICE = 5,    /* a device-side check failed (bad index, bad state)      */
    SGTP_E_UNSUPPORTED = 6
};

/* Limits of the library. */
#define SGTP_MAX_AGENTS 16        /* vehicles per race (so <= 15 opponents)         */
#define SGTP_MAX_T 128            /* horizon steps                                  */
#define SGTP_MAX_K (1 << 30)      /* samples per best response                      */

/* Planner parameters (Sec. IV-B names).  Passed by host pointer, copied at
 * call time. */
typedef struct sgtp_params {
    float dt;                     /* step [s]                                        */
    float wheelbase;              /* bicycle wheelbase [m]                           */
    float a_min, a_max;           /* acceleration limits of Pi_U [m/s^2]             */
    float delta_max;              /* |delta| <= delta_max of Pi_U [rad]              */
    float v_min, v_max;           /* speed clamp of the model [m/s]                  */
    float sigma_a, sigma_delta;   /* std-dev of the Gaussian perturbation (Sec. II)  */
    float Q[4];                   /* state weights over (x, y, psi, v) (Eq. ctrack)  */
    float R[2];                   /* control weights over (a, delta)                 */
    float S[2];                   /* control-rate weights over (a, delta)            */
    float w_game;                 /* weight of the game-aware cost (Eq. allc)        */
    float w_contest, w_long, w_block, w_safety;  /* Eqs. c_contest .. c_safety      */
    float s_contest;              /* contest range [m]                               */
    float s_role;                 /* blocking role gap [m]                           */
    float mu_tail;                /* tail share of the horizon for blocking          */
    float g_safe;                 /* desired separation [m]                          */
    float eps_alpha;              /* epsilon of the adaptive weight alpha            */
    float m_bd;                   /* required boundary clearance [m]                 */
    float d_col;                  /* collision distance [m]                          */
} sgtp_params;

/* ------------------------------------------------------------------ */
/* Raceline G (Sec. II, Preliminaries)                                  */
/* ------------------------------------------------------------------ */
typedef struct sgtp_track sgtp_track;   /* opaque, device resident, library owned */

/* Build a device raceline from HOST arrays.  xr: N x 4 waypoint states
 * (x, y, psi, v^r) of a CLOSED loop (waypoint N-1 joins waypoint 0); wl, wr:
 * N left/right widths (> 0).  3 <= N <= 1,048,576.  The library copies the
 * arrays, then a device kernel computes, per segment j, the chord to the
 * next waypoint, its squared-length inverse, the cumulative arc length s_j
 * and the width/heading/speed increments used by the linear reference maps
 * x^r(s), w^L(s), w^R(s).  Blocks until the track is ready.  On success
 * *out owns device memory released by sgtp_track_destroy. */
sgtp_status sgtp_track_create(const float *xr, const float *wl, const float *wr, int32_t N, void *stream,
                              sgtp_track **out);

/* Several racelines in one object (independent races of a batch): track t
 * holds waypoints offsets[t] .. offsets[t+1]-1 of the concatenated arrays.
 * offsets has n_tracks+1 HOST entries, offsets[0] = 0. */
sgtp_status sgtp_track_create_many(const float *xr, const float *wl, const float *wr, const int32_t *offsets,
                                   int32_t n_tracks, void *stream, sgtp_track **out);

void sgtp_track_destroy(sgtp_track *trk);

/* Host query: number of tracks, waypoints of track t, and its length (m). */
sgtp_status sgtp_track_info(const sgtp_track *trk, int32_t track_id, int32_t *n_tracks, int32_t *N, float *length);

/* ------------------------------------------------------------------ */
/* One best response (Alg. 1, one pass of the vehicle loop)             */
/* ------------------------------------------------------------------ */

/* Device scratch needed by sgtp_rollout_costs / sgtp_best_response. */
size_t sgtp_br_workspace_bytes(int32_t n_opp, int32_t T);

/* Per-sample cost, feasibility and violation of the K candidates of one
 * best response (Alg. 1: sampling, cost, feasibility indicator steps).
 *   x0        [4]                current state x_{i,t}
 *   u_nom     [T x 2]            nominal controls U-bar (Sec. II)
 *   vref_scale                   scale of the agent's reference speed (1 = raceline)
 *   opp       [n_opp x (T+1) x 4] fixed opponent predictions (may be NULL if n_opp = 0)
 *   game_on   0: cost = c_track only (the initial round of Alg. 1)
 *   cost, feasible, violation [K]  c (Eq. allc), h = b*o (Eq. selection), nu
 * Optional outputs (NULL to skip): states [K x (T+1) x 4], frenet
 * [K x (T+1) x 2] = (unwrapped progress s, lateral offset d) and controls
 * [K x T x 2] (the clipped samples).  0 <= n_opp <= SGTP_MAX_AGENTS-1,
 * 1 <= T <= SGTP_MAX_T, 1 <= K <= SGTP_MAX_K. */
sgtp_status sgtp_rollout_costs(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, const float *x0,
                               const float *u_nom, float vref_scale, const float *opp, int32_t n_opp, int32_t T,
                               int32_t K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                               int32_t game_on, float *cost, uint8_t *feasible, float *violation, float *states,
                               float *frenet, float *controls, void *workspace, size_t workspace_bytes,
                               void *stream);

/* The full best response: the same K candidates, then the selection of
 * Eq. selection with the least-violation fallback (ties to the lowest k),
 * and the re-rolled winner.
 *   k_star [1] (int32), u_star [T x 2], xi_star [(T+1) x 4], any_feasible [1]
 * All outputs are device pointers written on `stream`. */
sgtp_status sgtp_best_response(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, const float *x0,
                               const float *u_nom, float vref_scale, const float *opp, int32_t n_opp, int32_t T,
                               int32_t K, uint64_t seed, uint32_t race, uint32_t agent, uint32_t round,
                               int32_t game_on, int32_t *k_star, float *u_star, float *xi_star,
                               int32_t *any_feasible, void *workspace, size_t workspace_bytes, void *stream);

/* Scratch held by the library for sgtp_best_response_noalloc: the workspace
 * of the largest best response the ABI accepts (SGTP_MAX_AGENTS-1 = 15
 * opponents, T = SGTP_MAX_T = 128), 18 KiB. */
#define SGTP_NOALLOC_SCRATCH_BYTES 18432

/* sgtp_best_response without a caller-provided workspace (the paper has no
 * counterpart: this is an engineering entry point).  The scratch is one
 * statically allocated device array of SGTP_NOALLOC_SCRATCH_BYTES inside
 * the library, so the call never asks any allocator for memory.  It serves
 * callers that must not allocate while they run, for example a fixed-rate
 * vehicle controller that re-plans every control period (an allocation can
 * block for an unbounded time, and a failed one mid-race has no recovery),
 * and plain C hosts that have no device allocator of their own.
 *   - Arguments, outputs and results are those of sgtp_best_response.
 *   - The first call on each device looks up the scratch's device address
 *     (with that device current) and caches it; that lookup may initialise
 *     the CUDA context and load the library's module, so make the first
 *     call on a device before starting any stream capture.
 *   - Nothing in the scratch has to start at zero: every call rewrites all
 *     of it before reading it.
 *   - All calls on one device share the one scratch: calls that overlap in
 *     time (several streams, or several host threads without ordering)
 *     race on it and give wrong results.  Issue them on one stream, or
 *     order them with events.
 *   - A problem whose workspace (sgtp_br_workspace_bytes) exceeds
 *     SGTP_NOALLOC_SCRATCH_BYTES is rejected with SGTP_E_INVALID (the
 *     largest problem the ABI accepts fits, checked when the library is
 *     compiled).
 *   - The cached address lives as long as the process: after the device's
 *     context is destroyed (cudaDeviceReset) it is stale, so do not call
 *     this entry point on a device after resetting it. */
sgtp_status sgtp_best_response_noalloc(const sgtp_track *trk, int32_t track_id, const sgtp_params *p,
                                       const float *x0, const float *u_nom, float vref_scale, const float *opp,
                                       int32_t n_opp, int32_t T, int32_t K, uint64_t seed, uint32_t race,
                                       uint32_t agent, uint32_t round, int32_t game_on, int32_t *k_star,
                                       float *u_star, float *xi_star, int32_t *any_feasible, void *stream);

/* ------------------------------------------------------------------ */
/* The planning call (Alg. 1) and batches of independent races          */
/* ------------------------------------------------------------------ */

/* Launch shape of the persistent kernel.  Any zero field takes the
 * library's choice.  Every shape gives bit-identical results (each sample is
 * computed with the same code, and selection is an exact integer minimum).
 * Two families of builds:
 *   - 128-thread CTAs (3 per SM, 168 registers) rolling out one to three
 *     samples per thread at once, interleaved; the count is
 *     samples_per_thread, or, when 0, chosen per round as the fewest that
 *     put the round's samples in one wave of the grid (at most 3) -- for a
 *     round of several waves even at 3, 2 or 3, whichever pads K less to
 *     whole tiles, except a plain batch under the queue schedule (3);
 *   - 256-thread CTAs with one sample per thread: 3 per SM with 80
 *     registers, or (ctas_per_sm <= 2) 2 per SM with 128 registers.
 * Samples are processed in tiles of block x samples_per_thread consecutive
 * k (GA-IBR-MPPI: tiles of 256); a round whose samples fit the grid twice
 * over at one per thread takes half tiles, one sample for each thread of a
 * CTA's first half (the 128-thread build when samples_per_thread is 0, the
 * 256-thread builds always), so that its lone-sample chains spread over
 * twice the CTAs.  Defaults: a plain plan takes the
 * 128-thread build unless its Jacobi round holds at most 256 x SMs samples
 * (then 2 x 256 threads); a single learned-proposal plan takes the
 * 256-thread builds (2 per SM when its round has fewer 256-sample tiles than
 * 3 x SMs), a learned batch the 128-thread build; GA-IBR-MPPI takes the
 * 128-thread build with two samples per thread (a tile is then its 256
 * samples) unless its round is small, or the 256-thread builds with one. */
typedef struct sgtp_launch_opts {
    int32_t block;                /* threads per CTA: 128 or 256 (0: default)        */
    int32_t samples_per_thread;   /* 0 .. 3: samples each thread rolls out at once
                                     (> 1 only with block 128 or 0)                  */
    int32_t ctas_per_sm;          /* resident CTAs per SM (capped at the occupancy
                                     limit; default the limit)                       */
    int32_t window;               /* track segments staged in shared memory per CTA
                                     (rounded to a multiple of 4, at most 512)       */
    int64_t wait_timeout_ns;      /* limit of each device-side wait (default: 20 x the
                                     launch's work at 5e10 rollout-steps/s, >= 100 ms) */
    int32_t debug_flags;          /* SGTP_DEBUG_*; 0 in production                   */
    int32_t schedule;             /* SGTP_SCHEDULE_*; 0: default                     */
    int64_t *trace_ns;            /* optional DEVICE buffer of 3*L+8 int64: %globaltimer
                                     stamps by CTA 0 at the start, after setup, and after
                                     each round's proposal, sample and winner phases (under
                                     the queue schedule: when CTA 0 leaves each phase)    */
} sgtp_launch_opts;

/* How the rounds of a planning call are scheduled on the persistent grid.
 * LOCKSTEP: every CTA takes a fixed share of each round's sample tiles, then
 * of its winners, with a grid barrier after each phase (every race of a
 * batch waits for the slowest).  QUEUE: after the setup, CTAs claim work
 * items from one device queue (samples of round 0, winners of round 0,
 * samples of round 1, ...; with the learned proposal each round starts with
 * one proposal item per vehicle); a proposal or sample tile waits (bounded
 * by wait_timeout_ns) until its race's previous round is complete and, for
 * a tile, its vehicle's proposal is in; a winner waits until its vehicle's
 * tiles are in; so each race advances at its own pace.  Both give the same
 * plans bit for bit.  DEFAULT: QUEUE for batches, LOCKSTEP for single
 * races. */
#define SGTP_SCHEDULE_DEFAULT 0
#define SGTP_SCHEDULE_LOCKSTEP 1
#define SGTP_SCHEDULE_QUEUE 2

/* Fault injection for tests: CTA 0 never arrives at the grid barrier, so
 * every other CTA's wait runs out and the call reports SGTP_E_TIMEOUT in
 * status_dev.  No wait in the library is unbounded. */
#define SGTP_DEBUG_SKIP_BARRIER_ARRIVAL 1
/* Fault injection for tests, queue schedule: no winner item reports its
 * completion, so the next round's sample tiles wait until their limit and
 * the call reports SGTP_E_TIMEOUT. */
#define SGTP_DEBUG_SKIP_WINNER_SIGNAL 2

/* Description of one race of a batch (HOST array given to
 * sgtp_batch_create).  Arrays of a batch concatenate the races' agents:
 * race r owns agents agent_offset .. agent_offset + n_v - 1. */
typedef struct sgtp_race {
    int32_t track_id;             /* track of the sgtp_track object                  */
    int32_t n_v;                  /* vehicles, 1 .. SGTP_MAX_AGENTS                  */
    int32_t T;                    /* horizon, 1 .. SGTP_MAX_T                        */
    int32_t ego;                  /* ego vehicle index within the race               */
    uint32_t race_tag;            /* the `race` word of the noise counter            */
} sgtp_race;

typedef struct sgtp_batch sgtp_batch;   /* opaque, device resident, library owned */

/* Prepare a batch: validates the races, lays out the ragged arrays and
 * uploads the race table.  K samples per best response and L IBR rounds
 * are common to the batch.  Array sizes of sgtp_batch_plan follow from
 * sgtp_batch_sizes.  Blocks until the table is on the device. */
sgtp_status sgtp_batch_create(const sgtp_track *trk, const sgtp_race *races, int32_t n_races, int32_t K,
                              int32_t L, sgtp_batch **out);
void sgtp_batch_destroy(sgtp_batch *b);

/* Element counts of the batch arrays (any pointer may be NULL):
 *   agents  = sum n_v                     (X0 rows, vref_scale entries)
 *   u_elems = sum n_v * T * 2             (U_io)
 *   xi_elems= sum n_v * (T+1) * 4         (xi_out)
 *   ks      = sum ((L+1) * n_v + 1)       (k_star_out, round-major per race)
 *   workspace_bytes                       (device scratch of sgtp_batch_plan)
 * Race r's slices start at the prefix sums of these counts in race order. */
sgtp_status sgtp_batch_sizes(const sgtp_batch *b, int64_t *agents, int64_t *u_elems, int64_t *xi_elems,
                             int64_t *ks, size_t *workspace_bytes);

/* Plan every race of the batch in ONE persistent cooperative launch
 * (Alg. 1 per race):
 *   round 0: every vehicle answers the others' nominal rollouts (controls
 *            U_io, clipped) with w_game off -- the initialisation of Alg. 1
 *            with distance-based (collision-check) avoidance only;
 *   rounds 1..L: Jacobi best responses to the previous round;
 *   then one extra ego best response (round tag L+1).
 * After every best response the vehicle's nominal controls become the
 * selected ones.  Outputs: U_io (warm start for the next call), xi_out
 * (round-L trajectories; the ego's is its extra response), k_star_out.
 * Optional xi_hist / u_hist (NULL to skip) have (L+2) slots of xi_out /
 * U_io layout: slot r after round r, slot L+1 after the extra ego response.
 *   X0 [agents x 4], U_io [u_elems], vref_scale [agents], xi_out [xi_elems],
 *   k_star_out [ks] (int32), status_dev [1] (int32, written 0 or SGTP_E_*).
 * Workspace: workspace_bytes from sgtp_batch_sizes. */
sgtp_status sgtp_batch_plan(const sgtp_batch *b, const sgtp_params *p, const float *X0, float *U_io,
                            const float *vref_scale, uint64_t seed, float *xi_out, int32_t *k_star_out,
                            float *xi_hist, float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                            void *workspace, size_t workspace_bytes, void *stream);

/* Workspace of sgtp_ibr_plan. */
size_t sgtp_plan_workspace_bytes(int32_t n_v, int32_t T, int32_t L);

/* One race, the paper's planning call (Alg. 1; CT of Sec. IV-C covers all
 * of it).  Same semantics as sgtp_batch_plan with a single race whose
 * descriptor is passed by value, so no setup call is needed.
 *   X0 [n_v x 4], U_io [n_v x T x 2], vref_scale [n_v], xi_out
 *   [n_v x (T+1) x 4], k_star_out [(L+1)*n_v + 1], xi_hist/u_hist optional. */
sgtp_status sgtp_ibr_plan(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                          const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K, int32_t L,
                          int32_t ego, uint64_t seed, uint32_t race, float *xi_out, int32_t *k_star_out,
                          float *xi_hist, float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                          void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* GA-IBR-MPPI: the paper's second ablation (Sec. IV-A)                 */
/* ------------------------------------------------------------------ */
/* The same planning loop, samples, rollouts and game-aware cost as
 * sgtp_ibr_plan, but no feasibility selection: after each best response the
 * vehicle's nominal controls become the path-integral mean of its samples'
 * (clipped) controls, the update of standard MPPI,
 *     w_k = exp(-(c_k - c_min) / lambda),  U_new = sum_k w_k U^(k) / sum_k w_k,
 * with c_k the total cost (Eq. allc; round 0 without the game term), and
 * the response's trajectory is the rollout of U_new.  The paper gives no
 * temperature: lambda > 0 (in cost units) is an argument.  A sample whose
 * cost is not finite weighs nothing; if no sample of a response has a finite
 * cost, the clipped nominal is kept.  k_star_out receives each response's
 * lowest-cost sample (lowest k on ties), for inspection only.
 *   - Arrays, layouts, ownership, rounds and the status word are those of
 *     sgtp_ibr_plan; the workspace is sgtp_plan_mppi_workspace_bytes (it
 *     grows with K: one partial sum of 2T+2 floats per 256-sample tile).
 *   - Sums are formed in a fixed order (32-sample groups by warp shuffles,
 *     then groups, then tiles in index order, each tile's weights taken
 *     relative to its own minimum and rescaled by exp(-(m_t - c_min)/lambda)),
 *     so every launch shape gives bit-identical results.
 *   - SGTP_E_INVALID (nothing launched) for lambda not > 0 or not finite,
 *     and for the arguments sgtp_ibr_plan rejects. */
size_t sgtp_plan_mppi_workspace_bytes(int32_t n_v, int32_t T, int32_t L, int32_t K);

sgtp_status sgtp_ibr_plan_mppi(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                               const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                               int32_t L, int32_t ego, uint64_t seed, uint32_t race, float lambda, float *xi_out,
                               int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                               const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                               void *stream);

/* The same for every race of a batch in one launch (sgtp_batch_plan's
 * arrays); its workspace size comes from sgtp_batch_mppi_workspace_bytes. */
sgtp_status sgtp_batch_mppi_workspace_bytes(const sgtp_batch *b, size_t *workspace_bytes);

sgtp_status sgtp_batch_plan_mppi(const sgtp_batch *b, const sgtp_params *p, float lambda, const float *X0,
                                 float *U_io, const float *vref_scale, uint64_t seed, float *xi_out,
                                 int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                                 const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                 void *stream);

/* ------------------------------------------------------------------ */
/* Perturbed opponent predictions (robustness study, Table II)          */
/* ------------------------------------------------------------------ */
/* sgtp_ibr_plan / sgtp_batch_plan with every opponent prediction perturbed
 * before each best response uses it.  The paper's perturbation model is a
 * cited one that is not available; the perturbation here is Gaussian noise
 * in Frenet coordinates, to first order: predicted position p_tau (tau =
 * 1..T) of opponent j, as seen by vehicle i in round r, moves by
 * sigma_lon z_1 along the unit direction of p_tau's nearest raceline segment
 * and by sigma_lat z_2 along that direction's left normal, (z_1, z_2) the
 * Box-Muller pair of Philox counter (2^30 | j, (tau-1) >> 1, i | r << 16,
 * race) -- a counter no sample uses, since samples have k < 2^30.  The
 * prediction's progress gain moves by sigma_lon z_1 of tau = T and its
 * tail-mean offset by the mean of sigma_lat z_2 over the tail steps; the
 * opponent's current state is observed exactly.  With both sigmas 0 the
 * call equals the unperturbed one bit for bit.
 *   - Arguments, outputs, workspace (sgtp_plan_workspace_bytes /
 *     sgtp_batch_sizes) and errors as for sgtp_ibr_plan / sgtp_batch_plan.
 *   - SGTP_E_INVALID for a sigma that is negative or not finite. */
sgtp_status sgtp_ibr_plan_perturbed(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                    const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                    int32_t L, int32_t ego, uint64_t seed, uint32_t race, float sigma_lon,
                                    float sigma_lat, float *xi_out, int32_t *k_star_out, float *xi_hist,
                                    float *u_hist, int32_t *status_dev, const sgtp_launch_opts *opts,
                                    void *workspace, size_t workspace_bytes, void *stream);

sgtp_status sgtp_batch_plan_perturbed(const sgtp_batch *b, const sgtp_params *p, float sigma_lon, float sigma_lat,
                                      const float *X0, float *U_io, const float *vref_scale, uint64_t seed,
                                      float *xi_out, int32_t *k_star_out, float *xi_hist, float *u_hist,
                                      int32_t *status_dev, const sgtp_launch_opts *opts, void *workspace,
                                      size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* Closed-loop race simulation (receding horizon)                       */
/* ------------------------------------------------------------------ */
/* The evaluation setting of Sec. IV-A (trials of several vehicles that
 * re-plan every control period; metrics of the Evaluation Metrics
 * subsection), on the batch layout: every race of an sgtp_batch is one
 * trial.  A closed loop alternates sgtp_batch_plan (or _mppi) with
 * sgtp_sim_step on the same arrays; both only enqueue work, so the loop can
 * run on one stream and be captured in a CUDA graph.  Readings (the paper
 * races in a simulator with its own vehicle model and a cited pure-pursuit
 * tracker whose parameters it does not give):
 *   - the plant is the planner's kinematic bicycle (Sec. II) with the same
 *     float arithmetic, so replaying a plan's controls reproduces its
 *     trajectory exactly;
 *   - pure pursuit steers toward the planned position pp_preview steps
 *     ahead of the current substep (a time-based look-ahead):
 *     delta = clip(atan(2 wheelbase sin(alpha) / l_d)), alpha the bearing of
 *     the target relative to the heading, l_d its distance; the acceleration
 *     tracks the next planned speed, a = clip((v_plan - v) / dt);
 *   - the ego is in contact with an opponent when their reference points are
 *     closer than contact_dist, and with a wall when its boundary clearance
 *     min(w^R(s) + d, w^L(s) - d) drops below wall_margin; a trial ends at
 *     the ego's first contact or after max_steps control steps;
 *   - an opponent is in close interaction while |Delta s| < close_ds and
 *     |Delta d| < close_dd in Frenet coordinates (Delta s wrapped to the
 *     half lap); a segment is a maximal run of such steps. */
typedef struct sgtp_sim_params {
    int32_t n_apply;          /* control steps of each plan applied before re-planning, 1 .. min T */
    int32_t max_steps;        /* trial length in control steps                             */
    int32_t tracker;          /* SGTP_TRACK_CONTROLS or SGTP_TRACK_PURE_PURSUIT            */
    int32_t pp_preview;       /* pure pursuit: planned position this many steps ahead, >= 1 */
    float contact_dist;       /* vehicle contact distance between reference points (m)     */
    float wall_margin;        /* wall contact below this boundary clearance (m)            */
    float close_ds, close_dd; /* close-interaction box in Frenet coordinates (m)           */
} sgtp_sim_params;

#define SGTP_TRACK_CONTROLS 0        /* apply the plan's controls U_io[0 .. n_apply)       */
#define SGTP_TRACK_PURE_PURSUIT 1    /* track the planned trajectory xi by pure pursuit   */

/* Per-trial state and result, one per race, in DEVICE memory owned by the
 * caller (n_races x sizeof(sgtp_sim_race), 16-byte aligned); written by
 * sgtp_sim_reset and sgtp_sim_step, read by the caller after a stream sync.
 * Fields marked internal carry the loop's state between steps. */
typedef struct sgtp_sim_race {
    int32_t alive;             /* 1 while the trial runs                                  */
    int32_t steps;             /* control steps simulated (the trial duration / dt)      */
    int32_t ego_collision;     /* 0 none, 1 vehicle contact, 2 wall contact               */
    int32_t close_segments;    /* completed close-interaction segments, all opponents    */
    int32_t close_steps;       /* their total length in control steps                    */
    float ego_speed_sum;       /* sum of the ego's speed after every step                */
    float ego_du2_sum;         /* sum of ||u_k - u_{k-1}||^2 of the ego's applied controls */
    int32_t pad0;
    float progress[SGTP_MAX_AGENTS];   /* unwrapped Frenet progress gain s_t - s_0            */
    float rel0[SGTP_MAX_AGENTS];       /* s_{j,0} - s_{ego,0} wrapped to the half lap         */
    float d[SGTP_MAX_AGENTS];          /* Frenet offset after the last step                    */
    float s_raw[SGTP_MAX_AGENTS];      /* internal: last projection s in [0, L)               */
    int32_t close_run[SGTP_MAX_AGENTS]; /* internal: current close-interaction run            */
    float u_prev[2];                    /* internal: the ego's last applied control           */
    int32_t pad1[2];
} sgtp_sim_race;

/* Start every trial of the batch from the states X [agents x 4] (device):
 * projections of every vehicle, zero progress, alive = 1. */
sgtp_status sgtp_sim_reset(const sgtp_batch *b, const float *X, sgtp_sim_race *state, void *stream);

/* Advance every live trial by sp->n_apply control steps (fewer if the ego
 * makes contact): controls from U_io or by pure pursuit on xi (the plan's
 * xi_out layout), bicycle steps of all vehicles in lock step, projection of
 * every vehicle on the globally nearest segment after each step, contact and
 * close-interaction checks, metric sums.  X_io [agents x 4] receives the new
 * states and U_io [u_elems] the warm start shifted by the steps applied (the
 * last control repeated).  Trials that have ended are left untouched.
 * SGTP_E_INVALID (nothing launched) for sizes or parameters out of range. */
sgtp_status sgtp_sim_step(const sgtp_batch *b, const sgtp_params *p, const sgtp_sim_params *sp, float *X_io,
                          float *U_io, const float *xi, sgtp_sim_race *state, void *stream);

/* ------------------------------------------------------------------ */
/* CUDA graphs of planning calls                                        */
/* ------------------------------------------------------------------ */
typedef struct sgtp_graph sgtp_graph;   /* opaque, library owned */

/* Capture one sgtp_ibr_plan call (same arguments; captured on an internal
 * stream, nothing runs) into an instantiated CUDA graph.  Every pointer is
 * fixed in the graph: between launches the caller rewrites X0, U_io and
 * vref_scale in place (U_io also carries the warm start from the previous
 * launch).  Returns SGTP_E_CUDA if the driver refuses the capture. */
sgtp_status sgtp_graph_capture_plan(const sgtp_track *trk, int32_t track_id, const sgtp_params *p, int32_t n_v,
                                    const float *X0, float *U_io, const float *vref_scale, int32_t T, int32_t K,
                                    int32_t L, int32_t ego, uint64_t seed, uint32_t race, float *xi_out,
                                    int32_t *k_star_out, float *xi_hist, float *u_hist, int32_t *status_dev,
                                    const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                    sgtp_graph **out);

/* The same for one sgtp_batch_plan call. */
sgtp_status sgtp_graph_capture_batch(const sgtp_batch *b, const sgtp_params *p, const float *X0, float *U_io,
                                     const float *vref_scale, uint64_t seed, float *xi_out, int32_t *k_star_out,
                                     float *xi_hist, float *u_hist, int32_t *status_dev,
                                     const sgtp_launch_opts *opts, void *workspace, size_t workspace_bytes,
                                     sgtp_graph **out);

/* Change the noise seed of later launches (host-side update of the
 * instantiated graph; does not touch any stream). */
sgtp_status sgtp_graph_set_seed(sgtp_graph *g, uint64_t seed);

/* Launch the graph on `stream` (results as from the captured call). */
sgtp_status sgtp_graph_launch(sgtp_graph *g, void *stream);
void sgtp_graph_destroy(sgtp_graph *g);

/* ------------------------------------------------------------------ */
/* Measurement and verification (no paper counterpart)                 */
/* ------------------------------------------------------------------ */
/* FP32 FMA throughput of the current device, the peak the best-response
 * path's roofline is reported against: ctas_per_sm x SMs CTAs of 256
 * threads, each thread running eight independent chains of `iters` x 8
 * FMAs (packed != 0: the same count as fma.rn.f32x2 on four register
 * pairs).  Enqueues one launch on `stream`; `sink` is a device float array
 * of at least ctas_per_sm x SMs entries that is written only under a
 * condition no chain meets.  *flops (host) receives the launch's FLOP count
 * (2 per FMA); divide by its event-timed duration.  SGTP_E_INVALID for
 * ctas_per_sm outside [1, 8] or iters outside [1, 2^24]. */
sgtp_status sgtp_fma_probe(int32_t ctas_per_sm, int32_t iters, int32_t packed, float *sink, void *stream,
                           double *flops);

/* Raw Philox4x32-10 blocks of the noise (counter layout above), as the
 * sample loop computes them: block i (0 <= i < n) of counter
 * (k0 + i, c1, c2, c3) under key (seed lo32, seed hi32) into words[4 i ..
 * 4 i + 3] (DEVICE, n x 4 uint32).  The device also evaluates each block
 * with the key schedule computed round by round (the form the winner
 * re-roll uses) and adds the count of blocks where the two differ to
 * *mismatch (DEVICE int32, caller zeroes it).  One launch on `stream`. */
sgtp_status sgtp_philox_words(uint64_t seed, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, int32_t n,
                              uint32_t *words, int32_t *mismatch, void *stream);

/* The standard normal pairs (z_a, z_delta) the sample loop draws for
 * candidates k0 .. k0 + nk - 1 at steps 0 .. T-1 of best response (race,
 * agent, round) on noise stream stream_bit (0 plain, 1 proposal), FP32
 * Box-Muller on the words above: z[(i T + tau) 2 + {0, 1}] (DEVICE,
 * nk x T x 2).  One launch on `stream`. */
sgtp_status sgtp_noise_normals(uint64_t seed, uint32_t race, uint32_t agent, uint32_t round, uint32_t stream_bit,
                               uint32_t k0, int32_t nk, int32_t T, float *z, void *stream);

/* ------------------------------------------------------------------ */
/* Misc                                                                 */
/* ------------------------------------------------------------------ */
/* Wait for `stream` and read a device status word written by a planning
 * call (status_dev): *status_host receives 0 or the SGTP_E_* code of a
 * device-side failure (low byte) with flag bits above it.  Returns
 * SGTP_E_CUDA if the stream itself failed.  Blocks the calling thread. */
sgtp_status sgtp_sync_status(const int32_t *status_dev, void *stream, int32_t *status_host);

const char *sgtp_last_error(void);     /* thread-local text of the last failure */
const char *sgtp_version(void);
/* Number of kernel launches this library has enqueued since load (all
 * entry points); used to count launches inside a timed region. */
int64_t sgtp_launch_count(void);

/* Fault injection for tests (host side): the n-th device allocation the
 * library makes from now on (track, batch table, network, training scratch)
 * fails as if the device were out of memory, so that the entry point under
 * test returns SGTP_E_NOMEM after releasing what it had allocated; n <= 0
 * disarms.  Process-wide; no device work is involved. */
void sgtp_debug_fail_alloc(int32_t n);

#ifdef __cplusplus
}
#endif
#endif /* SGTP_H */
