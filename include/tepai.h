/*
 * tepai.h — C-ABI of the GB300 (sm_103a) MPS TE-PAI library (libtepai.so).
 *
 * Method: Hasselgren & Koczor, "Quantum-inspired classical simulation through
 * randomized time evolution" (arXiv 2604.13144).
 *
 * The library evolves an ensemble of independently sampled TE-PAI circuits.
 *   - Sampling (Sec. II.B protocol; App. A.3, Eq. settings / Eq. gammas):
 *     every rotation R_k(theta_kj) of the N-step product formula is replaced
 *     by I, R_k(sign(theta) Delta) or R_k(pi).
 *   - Evolution (Sec. II.A): each circuit is evolved as its own matrix product
 *     state, with two-site SVD updates truncated to chi_max / cutoff.
 *   - Measurement: <Z_i> at M snapshot steps.
 *   - Estimate (Sec. II.B; App. B): the signed, ||g(t)||_1-weighted ensemble
 *     mean.
 *
 * Conventions that hold for every call:
 *   - Host pointers are caller-owned. They are read or written only during
 *     the call and are never retained.
 *   - Device pointers (the tepai_dev_* calls) are also caller-owned, and must
 *     stay valid until the work queued on the given stream has completed.
 *   - The library allocates device memory only inside a tepai_ctx, which owns
 *     it until tepai_destroy.
 *   - Every call returns 0 (TEPAI_OK) or a TEPAI_ERR_* code; tepai_strerror
 *     names it. No C++ exception crosses this boundary.
 *   - Results depend only on (problem, params, seed, global sample index), not
 *     on the launch configuration.
 */
#ifndef TEPAI_H
#define TEPAI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define TEPAI_OK                    0
#define TEPAI_ERR_INVALID_ARG       1  /* n < 2, chi_max < 1, non-finite input, M does not divide steps ... */
#define TEPAI_ERR_THETA_EXCEEDS_DELTA 2 /* some |theta_k| > Delta, against the assumption of App. A.3 */
#define TEPAI_ERR_OUT_OF_MEMORY     3
#define TEPAI_ERR_CUDA              4  /* a CUDA runtime call failed; the CUDA error text is kept per thread */
#define TEPAI_ERR_NOT_CONVERGED     5  /* reserved: a Jacobi SVD that hits its sweep cap is counted in
                                          tepai_stats.n_not_converged and its result is still used */
#define TEPAI_ERR_WORKSPACE_TOO_SMALL 6
#define TEPAI_ERR_NO_DEVICE         7
#define TEPAI_ERR_DEVICE_CHECK      8  /* a kernel found a broken invariant (bond dimension out of range,
                                          non-finite norm); it stopped without touching memory out of
                                          bounds and the results of that launch are invalid */

/* ---- variants and precisions ----------------------------------------- */
#define TEPAI_UNBIASED 0  /* TE-PAI with settings A, B, C (App. A.3) */
#define TEPAI_NO_PI    1  /* biased TE-PAI without pi-rotations (Statement 3; App. A.4) */
#define TEPAI_TROTTER  2  /* deterministic first-order product formula (Eq. Trotter-Suzuki) */
#define TEPAI_CONTINUOUS 3 /* TE-PAI in the limit N -> infinity (App. A.3 at small theta, App. A.5,
                              Eq. overhead): term k fires B/C events as a Poisson process of rate
                              |c_k| (3 - cos Delta) / sin Delta; an event is C with probability
                              (1 - cos Delta) / (3 - cos Delta); ||g(t)||_1 =
                              exp(2 tan(Delta/2) ||c||_1 t). Needs 0 < Delta < pi. The evolved
                              time is T run_steps / n_steps; snapshot m is taken at that time
                              times m / n_snapshots, after every event at or before it. Event i
                              (from 0) of term k draws Philox4x64-10 counter (k, i, 1, 0) under
                              key (seed, sample): u = ((x0 >> 11) + 1) 2^-53 gives the waiting
                              time -ln(u) / rate, x1 < floor(P(C) 2^64) makes it C. Ties in time
                              go to the lower term index. */

#define TEPAI_FP64  0     /* all tensor arithmetic in FP64 */
#define TEPAI_MIXED 1     /* FP32 tensors and SVD; FP64 norms, truncation weights and reduction */

/* Spin chain / ring of Sec. III, Eq. (spinRing):
 * H = sum_i h_i Z_i + sum_b (Jx_b X X + Jy_b Y Y + Jz_b Z Z) on bond b = (b, b+1 mod n).
 * Term order within one Trotter step: Z_0..Z_{n-1}, then per bond XX, YY, ZZ. */
typedef struct {
    int n;                         /* number of spins, >= 2 */
    int periodic;                  /* 1 = ring (bond n-1 joins sites n-1 and 0) */
    const double *Jx, *Jy, *Jz;    /* host, length n (ring) or n-1 (chain) */
    const double *h;               /* host, length n */
    const unsigned char *init_bits;/* host, length n; initial product state, one code per site:
                                      0 |0>, 1 |1> (Z|0> = |0>), 2 |+>, 3 |->, 4 |+i>, 5 |-i> */
} tepai_problem;

typedef struct {
    double T;                      /* total evolution time of the product formula */
    long long n_steps;             /* N: theta_k = 2 c_k T / N (App. A.3) */
    double delta;                  /* Delta of setting B (Eq. settings) */
    long long n_samples;           /* N_s of this call */
    long long sample_offset;       /* global index of the first sample (shards use disjoint ranges) */
    long long run_steps;           /* steps actually evolved, 0 = all N */
    int chi_max;                   /* bond-dimension cap of every two-site update (Sec. II.A) */
    double cutoff;                 /* keep the fewest singular values whose discarded weight
                                      sum_{j>=k} s_j^2 <= cutoff * sum_j s_j^2 (then cap at chi_max) */
    int n_snapshots;               /* M; snapshot m after step m * run_steps / M, must divide */
    const int *obs_sites;          /* host, Z_i sites measured; NULL = all n */
    int n_obs;
    unsigned long long seed;       /* Philox4x64-10 key word 0 (key word 1 = global sample index) */
    int variant;                   /* TEPAI_UNBIASED | TEPAI_NO_PI | TEPAI_TROTTER | TEPAI_CONTINUOUS */
    int precision;                 /* TEPAI_FP64 | TEPAI_MIXED */
    int launch_variant;            /* 0 = built-in launch-shape rule. When the SVD working matrix is
                                      staged from global memory: 1 = two 256-thread CTAs per SM,
                                      2 = one 512-thread CTA per SM (both with the CUDA-core Jacobi
                                      passes), 7 = 256-thread CTAs running the Jacobi's Gram
                                      matrices and block updates and the theta and projection
                                      products on the tensor cores (TF32 operands split in two,
                                      FP32 accumulation; TEPAI_MIXED with chi_max <= 128; one CTA
                                      per SM, as for any kernel holding tensor memory, so only on
                                      request). When it fits in shared
                                      memory: 3, 4, 5, 6 = 64, 128, 256, 512 threads per CTA
                                      (smaller CTAs run more samples per SM). Variants that do not
                                      apply are ignored. tepai_autotune reports the fastest on this
                                      device. */
    const unsigned char *obs_strings; /* host, n_obs x n Pauli codes per site (0 I, 1 X, 2 Y, 3 Z):
                                      observable o is the string (x)_i P_{o,i}; NULL = Z on
                                      obs_sites. Values v[s][m][o] are <psi|P|psi>/<psi|psi>. */
    double tie_rel;                /* truncation ties (Sec. II.A keeps the largest singular values
                                      up to chi_max): a cut never splits a group of values whose
                                      neighbours lie within tie_rel * s_0 of each other; the whole
                                      group is discarded. 0 = the paper's rule, where only values
                                      equal to working precision (1e-12 s_0) are tied. A wider band
                                      (e.g. 1e-4) makes the kept state insensitive to rounding at
                                      nearly degenerate cuts, at the price of discarding them. */
    int three_site;                /* 1 = a two-site gate between chain positions p and p+2 (ring
                                      bonds in the folded order) is one three-site update: theta3 =
                                      A_p A_{p+1} A_{p+2} takes the gate on its outer physical
                                      indices and two truncated SVDs (2 d_p x 4 d_{p+3}, then
                                      2 k_1 x 2 d_{p+3}) split it back, each with the keep rule and
                                      renormalisation of a two-site update (Sec. II.A); the centre
                                      ends on p+2. 0 = swap routing (swap, gate, swap back: three
                                      truncated two-site updates). Each split counts as a gate update.
                                      The arena grows by 16 chi_max^2 values per CTA. */
} tepai_params;

/* Optional initial MPS shared by all samples (a "hybrid" start). Site tensors
 * A_p[d_p][2][d_{p+1}] are row-major, complex interleaved (re, im), and
 * concatenated over CHAIN positions p: natural site order for an open chain,
 * and for a ring the folded order 0, n-1, 1, n-2, 2, ... that the library
 * stores rings in (every ring bond within two chain positions). They need not
 * be normalised or canonical: every sample first brings them to right-canonical
 * form. */
typedef struct {
    const int *bond_dims;          /* length n+1, bond_dims[0] = bond_dims[n] = 1, each <= chi_max */
    const double *tensors;         /* host (tepai_run) or device (tepai_dev_*) */
} tepai_mps;

typedef struct {
    double events;                 /* non-identity gates applied (nu, summed over samples) */
    double gate_updates;           /* two-site SVD updates that apply a gate */
    double swap_updates;           /* two-site SVD updates of ring-bond routing */
    double qr_moves;               /* orthogonality-centre moves */
    double jacobi_sweeps;          /* summed over all SVDs */
    double max_discarded_weight;
    double alg_flops;              /* algorithmic real flops: 32 dl dc dr for each theta plus
                                      4 (14 mx mn^2 + 8 mn^3) for each SVD of an mx x mn matrix */
    int max_chi;
    int n_not_converged;
    int device_status[3];          /* first device check failure: (code, detail, CTA); code 0 =
                                      none, 1 bond dimension out of range, 2 invalid singular-value
                                      ranking, 3 non-finite column norm, 4 bulk copy did not land,
                                      5 Jacobi column handoff did not arrive, 6 invalid entry in
                                      the sample order, 7 tensor-core MMAs did not complete */
    double phase_cycles[8];        /* SM cycles per phase, summed over CTAs: init, sampler,
                                      single-site gates, theta, Jacobi SVD, truncation and
                                      write-back, centre moves (QR), measurement */
    int grid_ctas;                 /* CTAs of the ensemble launch */
    double jacobi_pairs;           /* column pairs examined by the Jacobi sweeps */
    double jacobi_rotations;       /* column pairs rotated by the Jacobi sweeps */
    double subphase_cycles[12];    /* SM cycles of parts nested in the phases above: Householder
                                      panels, trailing block-reflector updates, explicit Q, R times
                                      the neighbour site, SVD projection and write-back, waits on
                                      bulk copies, Jacobi passes, singular-value ranking; and inside
                                      the tensor-core Jacobi passes: Gram GEMMs, Gram assembly,
                                      rotation rounds, block updates with write-back */
    int sample_order;              /* 1 when the call handed out its samples costliest first
                                      (predicted two-site updates, from the sampler's own draws):
                                      sampled variants, more samples than CTAs, at most 65536
                                      draws per sample, unless TEPAI_LPT=0. Adds two small
                                      launches per call; results do not depend on it. */
    double seconds;                /* device time of the call's ensemble work (kernels of the
                                      last execute, CUDA events on its stream) */
    double mean_nu;                /* events / n_samples: mean non-identity gates per sample */
    double jacobi_reorth;          /* mixed precision: SVDs whose FP32 Jacobi stalled (rotation
                                      count not falling, or the sweep cap) and were finished by one
                                      pass with FP64 inner products and rotations */
    double tc_flops;               /* flops of the tensor-core MMAs issued (2 M N K per tcgen05.mma;
                                      a 3xTF32 product counts three), 0 on the CUDA-core paths */
    double three_site_updates;     /* bond-2 gates applied as three-site updates (two splits each) */
} tepai_stats;

/* Circuit event of one sample: Trotter step j (1-based), term k, setting v
 * (1 = B, 2 = C, 3 = deterministic Trotter gate). */
typedef struct { int32_t j; int32_t k; int32_t v; int32_t pad; } tepai_event;

typedef struct tepai_ctx tepai_ctx;

/* ---- context ---------------------------------------------------------- */
/* Create a context on CUDA device `cuda_device`, issuing work on `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream). */
int  tepai_create(tepai_ctx **out, int cuda_device, void *cuda_stream);
void tepai_destroy(tepai_ctx *ctx);

/* ---- host-buffer entry points (all buffers host memory) ---------------- */
/* Full run (Sec. II.B protocol steps 1-3). Outputs, each [M][n_obs] row-major:
 *   mean     ||g(t_m)||_1 * (1/N_s) sum_s sign_s,m v_s,m,i;
 *   stderr_  ||g(t_m)||_1 * sqrt(Var[v]/N_s) (Statement 2), may be NULL;
 *   partials [M][n_obs][3] = (Neumaier sum, compensation, sum of squares)
 *            of sign*v over this call's samples, so that shards can be merged;
 *            may be NULL.
 * `init` may be NULL (product state init_bits). stats may be NULL. */
int tepai_run(tepai_ctx *ctx, const tepai_problem *prob, const tepai_params *par,
              const tepai_mps *init, double *mean, double *stderr_, double *partials,
              tepai_stats *stats);

/* Per-sample values for parity checks: v [n_samples][M][n_obs] = <Z_i>/<psi|psi>
 * after step j_m, and sign [n_samples][M] = (-1)^{#C up to j_m} (App. B). */
int tepai_sample_values(tepai_ctx *ctx, const tepai_problem *prob, const tepai_params *par,
                        const tepai_mps *init, double *v, signed char *sign, tepai_stats *stats);

/* The events of global sample `sample`, drawn by the device sampler, in gate
 * order (j = step, from 1). For TEPAI_CONTINUOUS they come in time order and j
 * is the snapshot index m (from 1) of the first t_m at or after the event.
 * Writes min(count, cap) events to buf and the full count to *count. */
int tepai_export_circuit(tepai_ctx *ctx, const tepai_problem *prob, const tepai_params *par,
                         long long sample, tepai_event *buf, long long cap, long long *count);

/* Host planner only: g[m] = ||g(t_m)||_1 (App. A.6, finite-N product) and the
 * expected gate count per sample E[nu] = run_steps * sum_k q_k. For
 * TEPAI_CONTINUOUS: g[m] = exp(2 tan(Delta/2) ||c||_1 t_m) and
 * E[nu] = t_run sum_k rate_k (nu_inf of App. A.5 when run_steps = N); such
 * a problem is refused with TEPAI_ERR_INVALID_ARG when E[nu] > 1e7. */
int tepai_gnorm(const tepai_problem *prob, const tepai_params *par, double *g, double *expected_nu);

/* ---- device-resident entry points -------------------------------------- */
/* Bytes of device workspace for a call with at most `grid_ctas` CTAs
 * (0 = library default for this device). */
int tepai_dev_workspace_size(const tepai_problem *prob, const tepai_params *par,
                             int grid_ctas, size_t *bytes);
/* Plan on the host and upload the tables and the initial MPS (device
 * pointers in `init`, or NULL) into the caller's workspace, on `stream`. */
int tepai_dev_prepare(const tepai_problem *prob, const tepai_params *par, const tepai_mps *init,
                      void *d_workspace, size_t ws_bytes, int grid_ctas, void *stream);
/* Launch the ensemble on a prepared workspace: kernels only, no host
 * synchronisation, no allocation. Device outputs: d_mean/d_stderr [M][n_obs],
 * d_partials [M][n_obs][3], d_v [n_samples][M][n_obs], d_sign [n_samples][M]
 * (any may be NULL except d_mean). The first call captures its stream work
 * (counter zeroing, ensemble kernel, reduction, output copies) as a CUDA graph
 * and later calls replay it; a changed sample offset is written into the
 * captured kernel's arguments, and other output pointers or another stream
 * trigger a new capture. Environment TEPAI_GRAPHS=0 launches directly instead.
 * Calls on one workspace must not overlap. */
int tepai_dev_execute(void *d_workspace, double *d_mean, double *d_stderr, double *d_partials,
                      double *d_v, signed char *d_sign, void *stream);
/* Point a prepared workspace at another range of global sample indices
 * [offset, offset + n_samples): the next execute evolves those circuits. Host
 * bookkeeping only (no device work); the Philox key word 1 of sample s is s. */
int tepai_dev_set_sample_offset(void *d_workspace, long long sample_offset);
/* Copy the device statistics of the last execute on this workspace. Synchronises `stream`. */
int tepai_dev_stats(void *d_workspace, tepai_stats *stats, void *stream);
/* Forget a prepared workspace: frees its captured CUDA graph and its
 * bookkeeping (the caller still owns and frees the device memory). Calling it
 * on an unknown workspace is a no-op that returns TEPAI_OK. */
int tepai_dev_release(void *d_workspace);

/* Evolve ONE circuit (par->n_samples must be 1; the deterministic Trotter
 * variant gives the prefix of a hybrid run) from `init` (or the product state)
 * and return its final MPS in the tepai_mps layout: bond_dims[0..n] and the
 * site tensors concatenated over chain positions, complex interleaved, FP64,
 * normalised, in some mixed-canonical gauge. `capacity` is the size of
 * `tensors` in doubles; n * 2 * chi_max^2 * 2 always suffices. `*used`
 * receives the doubles written, and TEPAI_ERR_WORKSPACE_TOO_SMALL is returned
 * (nothing written to tensors) when capacity is short. The result can be
 * passed as the start state of later runs (Sec. IV hybrid: Trotter to t0,
 * TE-PAI after). */
int tepai_evolve_state(tepai_ctx *ctx, const tepai_problem *prob, const tepai_params *par,
                       const tepai_mps *init, int *bond_dims, double *tensors, long long capacity,
                       long long *used);

/* ---- launch-shape autotuner --------------------------------------------
 * Times every launch variant that applies to this problem on this device (see
 * tepai_params.launch_variant) on a short trial of the caller's own problem:
 * the same ring, precision and chi_max, one circuit per CTA, `trial_steps`
 * Trotter steps (0 = 1) from the given start state. Reports the fastest
 * variant and its rate in two-site updates per second of kernel time. The
 * trials use sample indices far above the caller's range and return no
 * estimates. Uses the context's stream and synchronises it. */
int tepai_autotune(tepai_ctx *ctx, const tepai_problem *prob, const tepai_params *par,
                   const tepai_mps *init, long long trial_steps, int *best_variant, double *best_rate);

/* ---- entry point without device allocation ------------------------------
 * The paper has no counterpart: this is a library-usage concern. Some callers
 * cannot allocate device memory: a host application that hands each
 * component a fixed device budget and forbids further allocations, a plug-in
 * that only receives buffers its framework allocated, or code that must not pay
 * cudaMalloc's implicit device synchronisation. This call runs the same
 * ensemble kernel as tepai_sample_values, from the product state init_bits,
 * with the same numerical settings, and allocates no device memory. All of its
 * scratch (tables, counters and one MPS arena per CTA) lives in a 64 MiB static
 * device array that every GPU loading the library holds until the process
 * exits. The host-side plan lives in static storage as well.
 *   d_v    [n_samples][M][n_obs] (double) and d_sign [n_samples][M] (int8):
 *          caller-owned device buffers (same layout as tepai_sample_values).
 *   stream cudaStream_t (NULL = legacy default stream). The call synchronises
 *          the stream and copies one status word back to the host before it
 *          returns.
 * Sizes: problems with at most 1024 spins; the MPS of one CTA must fit in the
 * array (n * 2 chi_max^2 + 8 chi_max^2 complex values), otherwise
 * TEPAI_ERR_WORKSPACE_TOO_SMALL. The number of CTAs is capped by what fits.
 * The first call on a device looks up the device address of the array
 * (cudaGetSymbolAddress) with that device current and keeps it; make that
 * first call before any stream capture, and do not call this entry point on a
 * device after cudaDeviceReset in the same process (the kept address would be
 * stale). Every call reuses the same array and leaves its contents behind;
 * each call clears its own counters. Calls serialise their host-side part, but
 * two calls whose GPU work overlaps (different streams or threads) race on the
 * array. */
int tepai_sample_values_static(const tepai_problem *prob, const tepai_params *par,
                               double *d_v, signed char *d_sign, void *stream);

/* ---- measured pipe throughput (roofline denominators) --------------------
 * No counterpart in the paper: a measurement helper. Runs three short
 * microbenchmarks on CUDA device `cuda_device` (each timed with CUDA events
 * after a warm-up launch, on a stream of its own) and reports TFLOP/s:
 *   fp32_tflops  FP32 fused multiply-add on every SM (8 independent chains per
 *                thread), the pipe of the Jacobi rotations and Householder QR;
 *   fp64_tflops  the same in FP64;
 *   tf32_tflops  tcgen05.mma kind::tf32 (M = 128, N = 256, K = 8) issued back
 *                to back by one thread per SM into TMEM, the pipe of the
 *                tensor-core Jacobi and products (a 3xTF32 product costs three).
 * Any output may be NULL (that benchmark is skipped). Allocates and frees a
 * few KB of device memory. Returns TEPAI_ERR_DEVICE_CHECK if the tensor-core
 * benchmark's bounded wait ran out. */
int tepai_measure_peaks(int cuda_device, double *fp32_tflops, double *fp64_tflops, double *tf32_tflops);

const char *tepai_strerror(int code);
/* Text of the last CUDA error seen by this thread ("" if none). */
const char *tepai_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TEPAI_H */
