/*
 * z2lgt.h -- C ABI of the GB300 (sm_103a) state-vector library for the
 * digital adiabatic simulation of quantum Z2 lattice gauge theory
 * (Cui, Shi, Yang, "Circuit-based digital adiabatic quantum simulation and
 * pseudoquantum simulation as new approaches to lattice gauge theory",
 * arXiv:1910.08020, JHEP 2020).
 *
 * Model (Sec. 2.1, and the "start from the ground state of X, H = X + K Z"
 * variant of Sec. 2.3 with K = s*lambda):
 *
 *     H(s) = -sum_l sigma^x_l - s * lambda * sum_p U_p,   U_p = prod_{l in p} sigma^z_l
 *
 * on a periodic d = 2 or 3 lattice with one qubit per link; the run starts in
 * |+>^N and ramps s = t/T linearly from 0 to 1 over M Trotter steps of
 * dt = T/M (Sec. 2.2: M = N_s * n, T = N_s * t_s, dt = t_s / n).
 *
 * Conventions shared by every call
 *   - qubit l is bit l of the amplitude index; sigma^z|0> = |0>,
 *     sigma^z|1> = -|1> (Sec. 2.1);
 *   - site s = x + L_x (y + L_y z); link l(s, mu) = d*s + mu (mu = 0: +x,
 *     1: +y, 2: +z); plaquette (s, mu < nu) = {l(s,mu), l(s+mu,nu),
 *     l(s+nu,mu), l(s,nu)}, listed site-major then plane (01, 02, 12);
 *     star(s) = {l(s,mu), l(s-mu,mu)};
 *   - a state is 2^N amplitudes, interleaved (re, im), in DEVICE memory:
 *     Z2_C64 = 2 x float (8 B per amplitude), Z2_C128 = 2 x double (16 B);
 *     the buffer must be 256-byte aligned and is owned by the caller (the
 *     library never frees caller memory); every state operation is in place;
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream); calls
 *     enqueue work on it and, unless stated otherwise, return before the GPU
 *     finishes; calls that return host results synchronise that stream;
 *   - every call returns Z2_OK (0) or a negative Z2_ERR_* code; the message
 *     of the last error on a context is z2_last_error(ctx).  No C++
 *     exception, abort or exit crosses this interface.
 *   - a context is used by one host thread at a time.
 */
#ifndef Z2LGT_H
#define Z2LGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define Z2_OK 0
#define Z2_ERR_ARG (-1)            /* invalid argument (NULL, size, range)          */
#define Z2_ERR_LATTICE (-2)        /* lattice not supported (d, L, qubit count)     */
#define Z2_ERR_OOM (-3)            /* device or host allocation failed              */
#define Z2_ERR_BUDGET (-4)         /* request exceeds the server's HBM budget       */
#define Z2_ERR_CUDA (-5)           /* a CUDA runtime call failed                    */
#define Z2_ERR_DEVICE_TIMEOUT (-6) /* a bounded device-side wait gave up            */
#define Z2_ERR_CANCELLED (-7)      /* the request was cancelled                     */
#define Z2_ERR_NOT_FOUND (-8)      /* unknown server ticket                         */

/* ---- enumerations --------------------------------------------------------- */
#define Z2_FIRST_ORDER 0 /* Eq. (a): per step psi <- R(dt) D(lambda s_j dt) psi            */
#define Z2_SYMMETRIC 1   /* Eq. (s): psi <- D(lambda s_j dt/2) R(dt) D(lambda s_{j-1} dt/2) psi */

#define Z2_C64 0  /* complex64 state, FP32 arithmetic, FP64 angles and reductions */
#define Z2_C128 1 /* complex128 state, FP64 throughout                            */

#define Z2_SAMPLE_STD 0   /* symmetric halves at s_{j-1} and s_j (second order)              */
#define Z2_SAMPLE_PAPER 1 /* both halves at s_j: the literal right-end rule of Sec. 2.2 (O(dt)) */

/* mask kinds for z2_lattice_masks (bit l set = link l in the operator) */
#define Z2_MASK_PLAQ 0       /* U_p, one per plaquette (Sec. 2.1)                         */
#define Z2_MASK_STAR 1       /* Gauss-law G_s, one per site (Sec. 2.1)                    */
#define Z2_MASK_WILSON_2X2 2 /* 2x2 loop at the origin, xy plane (XOR of its 4 plaquettes) */
#define Z2_MASK_CONTOUR 3    /* contours c1, c2, c3: perimeters 4, 6, 8 (Sec. 3.1)        */
#define Z2_MASK_W_MU 4       /* non-contractible Wilson lines W_mu, one per direction     */
#define Z2_MASK_V_MU 5       /* 't Hooft operators V_mu: mu-links of the plane x_mu = 0   */

/* z2_results.flags bits */
#define Z2_FLAG_WILSON_DEGENERATE (1u << 0)  /* 2x2 loop wraps the torus: NaN reported */
#define Z2_FLAG_CONTOUR_DEGENERATE (1u << 1) /* some contour wraps: NaN reported        */
#define Z2_FLAG_NO_FIDELITY (1u << 2)        /* no reference state given: NaN           */

/* sizes of the fixed arrays in z2_results */
#define Z2_MAX_LINKS 34
#define Z2_MAX_PLAQ 32
#define Z2_MAX_SITES 32

typedef struct z2_ctx z2_ctx;
typedef struct z2_lattice z2_lattice;
typedef struct z2_server z2_server;

typedef struct {
    int32_t d, L[3];
    int32_t n_links; /* N = qubits = d * prod L  (Sec. 2.1)   */
    int32_t n_plaq;  /* N_p = N (d - 1) / 2       (Sec. 2.1)  */
    int32_t n_sites;
} z2_lattice_info;

/* Parameters of one adiabatic run (Sec. 2.2 and 2.3).  Caller-owned. */
typedef struct {
    double lambda;     /* coupling of the plaquette term at s = 1 (K = 1/g of Sec. 2.3) */
    double T;          /* total evolution time (T = N_s t_s)                            */
    int32_t M;         /* number of Trotter steps (M = N_s n), >= 1                     */
    int32_t decomp;    /* Z2_FIRST_ORDER or Z2_SYMMETRIC                                */
    int32_t precision; /* Z2_C64 or Z2_C128                                             */
    int32_t sampling;  /* Z2_SAMPLE_STD or Z2_SAMPLE_PAPER                              */
} z2_run_params;

/* Observables of a state (Sec. 2.4), reductions in FP64.  Caller-owned.
 * Expectation values are <psi|O|psi> / <psi|psi> and the fidelity is
 * |<ref|psi>|^2 / (<ref|ref> <psi|psi>); `norm` is <psi|psi> as measured
 * (1 up to rounding).  Arrays are filled up to n_plaq / n_sites / n_links / d
 * entries. */
typedef struct {
    double s;                       /* ramp parameter the energy refers to         */
    double energy;                  /* <H(s)> = -sum<sigma^x_l> - s lambda sum<U_p>
                                       (the z2_*_gramp calls: <H(g)>, see there)  */
    double norm;                    /* <psi|psi>                                   */
    double mean_plaq;               /* mean <U_p>                                  */
    double wilson_2x2;              /* <W> of the 2x2 loop (NaN if degenerate)     */
    double mean_star;               /* mean Gauss-law <G_s> (exactly 1 in theory)  */
    double fidelity;                /* normalised |<ref|psi>|^2 (NaN without ref)  */
    double plaq[Z2_MAX_PLAQ];       /* <U_p>                                       */
    double star[Z2_MAX_SITES];      /* <G_s>                                       */
    double sigmaz[Z2_MAX_LINKS];    /* <sigma^z_l>                                 */
    double sigmax[Z2_MAX_LINKS];    /* <sigma^x_l>                                 */
    double wmu[3];                  /* <W_mu>                                      */
    double vmu[3];                  /* <V_mu>                                      */
    double contours[3];             /* <W_c1>, <W_c2>, <W_c3>                      */
    uint32_t flags;                 /* Z2_FLAG_* bits                              */
    int32_t status;                 /* Z2_OK or the error of this run (batches)    */
} z2_results;

/* ---- context --------------------------------------------------------------
 * A context binds one CUDA device and owns the library's device scratch
 * (reduction partials, phase tables) and its cached execution plans. */
int z2_ctx_create(int device, z2_ctx **out);
int z2_ctx_destroy(z2_ctx *ctx);
/* Message of the last failed call on ctx (ctx may be NULL for the last
 * failure of z2_ctx_create / z2_lattice_create on this thread).  The string
 * is owned by the library and valid until the next call on ctx. */
const char *z2_last_error(const z2_ctx *ctx);
/* Library version string (static storage). */
const char *z2_version(void);

/* Number of kernel launches this context has issued so far (all calls). */
int z2_ctx_launch_count(const z2_ctx *ctx, uint64_t *out);
/* Drop every cached execution plan (phase tables and pass lists); the next
 * call rebuilds and re-uploads what it needs.  Synchronises the device. */
int z2_ctx_flush_plans(z2_ctx *ctx);

/* Execution options of a context (they change how, not what, is computed).
 * Setting one drops the cached plans. */
#define Z2_OPT_TILE_BITS 0    /* 0 = automatic, else amplitudes per tile = 2^value (8..14)   */
#define Z2_OPT_PASS_VARIANT 1 /* 0 = automatic (as 5 where it applies, else 3, else 1),
                                 1 = direct global loads, 2 = TMA per CTA,
                                 3 = TMA ring (several tiles per CTA, complex64, multi-tile),
                                 4 = TMA ring with 32 pairs per thread (tile bits 12..13),
                                 5 = TMA ring, strided groups with 32 pairs per thread and
                                     the low group with 16 (tile bits 12..13)               */
#define Z2_OPT_SPLIT_LOW_BITS 2 /* ring plans with two strided groups: how many of the split
                                   group's bits sit at the bottom of the strided range (the
                                   rest at the top); 0 = automatic (share the rotated bits
                                   below bit 21 evenly between the groups), 1..8 = that many */
#define Z2_OPT_GANG_WAIT_POLLS 3 /* Z2_SWEEP_PERSISTENT: polls of a gang barrier (a counter in
                                    global memory) before the kernel gives up, sets the device
                                    error flag and returns, so the call reports
                                    Z2_ERR_DEVICE_TIMEOUT; 0 = the default (2^26 polls with a
                                    short sleep each).  A small value makes the bounded wait
                                    run out on purpose, to exercise the error path. */
int z2_ctx_set_option(z2_ctx *ctx, int32_t option, int32_t value);

/* Autotuner: times each candidate execution plan of `lat` at `precision`
 * (tile sizes x kernel variants; the tile size fixes how many qubits one pass
 * fuses) on a few Trotter steps of `state` (a device state of that lattice
 * and precision; its contents are overwritten), keeps the fastest for that
 * qubit count and precision in the context (used when no explicit option is
 * set) and, if the environment variable Z2_TUNE_CACHE names a file, records
 * it there for later contexts.  Synchronises `stream`. */
typedef struct {
    int32_t tile_bits;     /* chosen tile size (qubits per tile)              */
    int32_t variant;       /* chosen Z2_OPT_PASS_VARIANT value                */
    double us_per_step;    /* measured time of one Trotter step               */
    int32_t n_candidates;  /* candidates timed                                */
} z2_tune_result;
int z2_autotune(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, void *stream,
                z2_tune_result *out);

/* ---- lattice (Sec. 2.1) ---------------------------------------------------
 * d in {2, 3}; each L_mu >= 2; N = d * prod(L) <= Z2_MAX_LINKS and fits the
 * device.  Periodic boundaries only.  Host-only objects. */
int z2_lattice_create(int32_t d, const int32_t *L, z2_lattice **out);
int z2_lattice_destroy(z2_lattice *lat);
int z2_lattice_info_get(const z2_lattice *lat, z2_lattice_info *out);
/* Copies the masks of `kind` into out[0 .. cap), count in *n.  Returns
 * Z2_ERR_ARG if cap is too small (then *n still holds the count). */
int z2_lattice_masks(const z2_lattice *lat, int32_t kind, uint64_t *out, size_t cap, size_t *n);
/* Bytes of a state of this lattice at `precision`. */
int z2_state_bytes(const z2_lattice *lat, int32_t precision, size_t *bytes);

/* ---- state preparation and the two layers of a step ---------------------- */
/* psi <- |+>^N, every amplitude 2^{-N/2} (Sec. 2.3, ground state of X). */
int z2_init_plus(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, void *stream);
/* psi <- D(theta) psi, D(theta) = exp(i theta sum_p U_p): the whole plaquette
 * layer as one diagonal pass (Eq. (ara) applied to every plaquette, Sec. 2.2). */
int z2_apply_plaquettes(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state,
                        double theta, void *stream);
/* psi <- R(dt) psi, R(dt) = prod_l exp(i dt sigma^x_l) = prod_l R_x^l(-2 dt):
 * the transverse-field layer (Sec. 2.2). */
int z2_apply_rx_layer(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state,
                      double dt, void *stream);
/* psi <- H^{(x)N} psi (Hadamard on every qubit): maps sigma^x-type operators
 * to sigma^z-type ones, "H sigma^z H" of Sec. 2.4.  Its own inverse. */
int z2_apply_hadamard(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state,
                      void *stream);

/* ---- evolution (Sec. 2.2) -------------------------------------------------
 * Applies steps j0+1 .. j1 (0 <= j0 <= j1 <= M) of the schedule of `p` to
 * `state` in place.  A whole run is j0 = 0, j1 = M; cutting a run into
 * segments is the paper's pause-measure-resume (Sec. 2.4) and equals the
 * uncut run up to rounding.  Symmetric segments close with the half layer
 * D(lambda s_{j1} dt / 2), so the state is at s = j1/M on return. */
int z2_evolve(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state, int32_t j0,
              int32_t j1, void *stream);

/* Shape of the execution plan z2_evolve uses for steps j0+1 .. j1: the
 * qubits are split into n_groups groups of at most tile_bits qubits; each
 * streaming pass over the state applies one group's gates (and at a step
 * boundary the plaquette layer between two applications of the same group),
 * so a step costs n_groups - 1 passes (1 when n_groups == 1, where the whole
 * state is one tile and the run is a single launch). */
typedef struct {
    int32_t tile_bits;      /* qubits held by one CTA tile                   */
    int32_t n_groups;       /* qubit groups                                  */
    int32_t n_passes;       /* streaming passes over the state               */
    int32_t n_launches;     /* kernel launches of the segment                */
    int32_t n_tables;       /* phase tables (one per plaquette layer)        */
    int32_t flip;           /* 1 if a final all-qubit sigma^x flip is applied */
    int32_t low_tile_bits;  /* tile of the low (contiguous) group's passes:
                               tile_bits, or one less where the complex64
                               ring runs that group on twice the workers    */
} z2_plan_info;
int z2_evolve_plan_info(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, int32_t j0, int32_t j1,
                        z2_plan_info *out);

/* Host-only view of the qubit grouping a plan uses (the streaming passes of
 * Sec. 2.3's layers, see z2_plan_info): for a state of n_qubits at
 * `precision`, with tile size `tile_bits` (0 = automatic) and pass variant
 * `variant` (Z2_OPT_PASS_VARIANT values), writes up to max_groups groups, the
 * low (contiguous) group first.  Group i rotates global bits [b, b + k1) and,
 * when k1 < k, also [b2, b2 + k - k1) (a group split in two ranges, the upper
 * one ending at bit n_qubits - 1); its tiles hold 2^tile_bits amplitudes, the
 * c lowest global bits followed by the group's bits.  assume_tma != 0 plans as
 * if the driver's tensor-map encoder were available (the TMA ring plans), so
 * that the grouping can be inspected on any machine.  Needs no GPU and
 * allocates nothing on the device.  Errors: Z2_ERR_ARG, Z2_ERR_LATTICE (no
 * tile size fits). */
typedef struct {
    int32_t tile_bits;  /* tile size of this group's passes                     */
    int32_t c;          /* passenger bits: global bits [0, c) in every tile     */
    int32_t b;          /* first rotated global bit                             */
    int32_t k;          /* rotated bits                                         */
    int32_t k1;         /* rotated bits starting at b (k1 == k: contiguous)     */
    int32_t b2;         /* start of the upper range when k1 < k, else 0         */
} z2_group_info;
int z2_plan_geometry(int32_t n_qubits, int32_t precision, int32_t tile_bits, int32_t variant, int32_t assume_tma,
                     z2_group_info *groups, int32_t max_groups, int32_t *n_groups);

/* ---- observables (Sec. 2.4) -----------------------------------------------
 * Fills `out` for the state at ramp parameter s (energy = <H(s)>).  `ref` is
 * an optional device state of the same size and precision for the fidelity
 * |<ref|psi>|^2 (NULL: NaN and Z2_FLAG_NO_FIDELITY).  sigma^x-type
 * quantities are measured as sigma^z after a Hadamard layer, which is undone
 * before return, so `state` is unchanged up to rounding.  Synchronises
 * `stream`. */
int z2_measure(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state, double s,
               const void *ref, void *stream, z2_results *out);
/* Whole run: z2_init_plus, z2_evolve(0, M), z2_measure(s = 1). */
int z2_run(z2_ctx *ctx, const z2_lattice *lat, const z2_run_params *p, void *state,
           const void *ref, void *stream, z2_results *out);

/* ---- raw reductions (Sec. 2.4) --------------------------------------------
 * out[k] = sum_i |psi_i|^2 (-1)^{popcount(i & masks[k])} = <prod_{l in mask_k} sigma^z_l>
 * for k < n_masks (host arrays), in FP64.  Synchronises `stream`. */
int z2_zsums(z2_ctx *ctx, int32_t n_qubits, int32_t precision, const void *state,
             const uint64_t *masks, int32_t n_masks, double *out, void *stream);
/* Densities of states (Sec. 3.3, the histograms of the Z and X terms).
 * Z2_DOS_Z: out[k] = sum of |psi_i|^2 over the basis states with exactly k
 *   plaquettes of U_p = -1, k = 0..n_plaq (so <sum_p U_p> = sum_k (N_p - 2k)
 *   out[k]).
 * Z2_DOS_X: the same in the sigma^x basis, binned by the number w of links
 *   with sigma^x = -1, w = 0..n_links (X = -sum_l sigma^x_l = 2w - n_links).
 *   The state is taken to that basis by a Hadamard layer and back (Sec. 2.4),
 *   so it is unchanged up to rounding.
 * `out` (host) must hold cap >= n_plaq + 1 (Z) or n_links + 1 (X) doubles;
 * *n_bins receives the count.  FP64 sums, bit-reproducible for a given size.
 * Synchronises `stream`.  Errors: Z2_ERR_ARG (NULL, bad kind or precision,
 * cap too small, unaligned state), Z2_ERR_CUDA, Z2_ERR_DEVICE_TIMEOUT. */
#define Z2_DOS_Z 0
#define Z2_DOS_X 1
int z2_dos(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, void *state, int32_t kind, double *out,
           int32_t cap, int32_t *n_bins, void *stream);
/* out[0] + i out[1] = <a|b> = sum_i conj(a_i) b_i, FP64.  Synchronises `stream`. */
int z2_overlap(z2_ctx *ctx, int32_t n_qubits, int32_t precision, const void *a, const void *b,
               double *out, void *stream);

/* ---- the paper's own schedule (Sec. 2.2-2.4, Sec. 4.3) ---------------------
 * The paper ramps H(g) = Z + g X, Z = -sum_p U_p, X = -sum_l sigma^x_l, from
 * g = 0 upward, starting in the ground state of Z.  The ramp has N_s steps of
 * n substeps; substep m of step k runs for t_s / n at
 * g_{k,m} = (k - 1) g_s + m g_s / n (Sec. 2.2), split as
 * exp(-i Z t_s/n) exp(-i g X t_s/n) (Z2_FIRST_ORDER: the paper's asymmetric
 * split, Eq. (a), the X factor acting first) or exp(-i Z t_s/2n)
 * exp(-i g X t_s/n) exp(-i Z t_s/2n) (Z2_SYMMETRIC, Eq. (s)).  The same fused
 * passes as z2_evolve run it: the plaquette angle is fixed and every
 * transverse-field layer has its own angle g_{k,m} t_s / n.  Caller-owned. */
typedef struct {
    double g_s;        /* increase of g per step                          */
    double t_s;        /* time per step                                   */
    int32_t N_s;       /* steps, >= 1 (N_s * n <= 2^24)                   */
    int32_t n;         /* substeps per step, >= 1                         */
    int32_t decomp;    /* Z2_FIRST_ORDER (Eq. a) or Z2_SYMMETRIC (Eq. s)  */
    int32_t precision; /* Z2_C64 or Z2_C128                               */
} z2_gramp_params;

/* The start state of Sec. 2.4: prod_p P_p |+>^N normalised, P_p = (1 + U_p)/2,
 * i.e. the equal superposition of every link configuration with all U_p = +1
 * (the ground state of Z, with G_s = V_mu = +1), multiplied by W_mu for every
 * bit mu set in `sectors` (bit 0 = x, 1 = y, 2 = z): the degenerate ground
 * state of Z in another topological sector, whose V_nu flip sign where the
 * loop of W_mu crosses their surface (Sec. 2.4, Sec. 4.3).  Built without a
 * projection: 2^{-r/2} on the r-dimensional GF(2) span of the plaquette
 * masks (shifted by the W_mu masks), then the Hadamard layer.  Enqueued on
 * `stream`.  Z2_ERR_ARG for sector bits >= d. */
int z2_init_projected(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, uint32_t sectors, void *state,
                      void *stream);
/* Steps k0+1 .. k1 of the ramp (0 <= k0 <= k1 <= N_s), in place, enqueued on
 * `stream`; segments compose: (0, a) then (a, b) equals (0, b). */
int z2_evolve_gramp(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, void *state, int32_t k0,
                    int32_t k1, void *stream);
/* Observables as z2_measure, except out->s = g and
 * out->energy = <H(g)> = -sum_p <U_p> - g sum_l <sigma^x_l>.  Synchronises
 * `stream`.  The state is unchanged. */
int z2_measure_gramp(z2_ctx *ctx, const z2_lattice *lat, int32_t precision, double g, void *state, const void *ref,
                     void *stream, z2_results *out);
/* z2_init_projected(sectors), all N_s steps, z2_measure_gramp at g = N_s g_s. */
int z2_run_gramp(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, uint32_t sectors, void *state,
                 const void *ref, void *stream, z2_results *out);

/* ---- gate-level circuits (Sec. 2.3, Eq. (ara), Figs. 3 and 4) --------------
 * One launch per gate on a state of n_qubits qubits (qubit q = index bit q),
 * the way the paper's simulator executed its circuits: for a literal
 * comparison with the fused passes and with the paper's gate counts, not for
 * speed.  Gates: Z2_GATE_CNOT flips q1 where q0 is 1; Z2_GATE_RZ is
 * R_z(angle) = exp(-i angle sigma^z / 2) on q0; Z2_GATE_RX is
 * R_x(angle) = exp(-i angle sigma^x / 2) on q0; Z2_GATE_H is the Hadamard
 * gate on q0 (angle ignored).  Enqueued on `stream`. */
#define Z2_GATE_CNOT 0
#define Z2_GATE_RZ 1
#define Z2_GATE_RX 2
#define Z2_GATE_H 3
int z2_apply_gate(z2_ctx *ctx, int32_t n_qubits, int32_t precision, void *state, int32_t kind, int32_t q0,
                  int32_t q1, double angle, void *stream);
/* Steps k0+1 .. k1 of the paper's ramp (z2_gramp_params) gate by gate, on a
 * state of N + 1 qubits whose top qubit (bit N) is the ancilla, in |0>.
 * Every substep applies, in the paper's order, the transverse-field factor as
 * N single-link gates R_x(-2 g_{k,m} t_s / n) and each plaquette factor
 * exp(-i Z_p tau) as the ancilla circuit of Eq. (ara): a CNOT from each of its
 * four links onto the ancilla, R_z(-2 tau) on the ancilla, the four CNOTs
 * again in reverse order (9 gates; tau = t_s/n, or t_s/2n twice in the
 * symmetric split, unmerged).  The ancilla returns to |0>, so the links' half
 * of the state equals what z2_evolve_gramp gives.  *n_gates (optional) = the
 * gates applied: (k1 - k0) n (N + 9 N_p) first order, (k1 - k0) n (N + 18 N_p)
 * symmetric.  Enqueued on `stream`. */
int z2_evolve_gramp_circuit(z2_ctx *ctx, const z2_lattice *lat, const z2_gramp_params *gp, void *state, int32_t k0,
                            int32_t k1, void *stream, uint64_t *n_gates);

/* ---- phase estimation (Sec. 2.4, Eq. (leap), Fig. 5) ------------------------
 * The controlled evolution U(t) = |0><0| (x) exp(-iHt) + |1><1| (x) exp(iHt)
 * for H = Z + g X at fixed g, with exp(-iHt) by n Trotter steps of t/n,
 * (exp(-i Z t/n) exp(-i g X t/n))^n (Z2_FIRST_ORDER) or
 * (exp(-i Z t/2n) exp(-i g X t/n) exp(-i Z t/2n))^n (Z2_SYMMETRIC).  The
 * control is an ancilla that chooses the direction of time.  Caller-owned. */
typedef struct {
    double g;          /* transverse coupling, fixed                      */
    double t;          /* evolution time of the |0> branch (-t for |1>)   */
    int32_t n;         /* Trotter steps, 1 .. 2^24                        */
    int32_t decomp;    /* Z2_FIRST_ORDER or Z2_SYMMETRIC                  */
    int32_t precision; /* Z2_C64 or Z2_C128                               */
    int32_t reserved;  /* 0                                               */
} z2_qpe_params;
/* U(t) in place on a state of N + 1 qubits whose top qubit (bit N) is the
 * control: its first 2^N amplitudes (control |0>) evolve for +t, the next
 * 2^N for -t, each with the fused passes of z2_evolve.  For an eigenstate
 * |u> of H, (|0> + |1>)|u>/sqrt(2) becomes (e^{-iEt}|0> + e^{iEt}|1>)|u>/sqrt(2):
 * z2_overlap of the two halves (n_qubits = N) then reads e^{2iEt}/2.
 * Enqueued on `stream`. */
int z2_controlled_evolution(z2_ctx *ctx, const z2_lattice *lat, const z2_qpe_params *qp, void *state, void *stream);

/* ---- allocation-free reduction ----------------------------------------------
 * The paper has no counterpart to this call: it serves callers that cannot
 * allocate device memory (a process under a hard memory cap, a plug-in that
 * is handed a fixed arena, code that must not call cudaMalloc once running).
 * It computes what z2_zsums does without a context and without allocating:
 * its scratch is a fixed 256 KB array inside the library (1024 x 32 partial
 * sums and 32 results, doubles), held on every GPU that loads the library
 * until the process exits.  Limits: 1 <= n_masks <= 32 (larger counts return
 * Z2_ERR_ARG with a message in z2_last_error(NULL)), 8 <= n_qubits <= 34.
 * Each thread sums runs of 16 amplitudes in the state's precision and adds
 * each run into FP64; everything after that (warps, blocks, the final sum) is
 * FP64.  z2_zsums adds in another order, so the two agree within 1e-6
 * (complex64) or 1e-12 (complex128), not bit for bit.  The first call on a
 * device (and again after the device's context changes, e.g. after
 * cudaDeviceReset) looks up the array's device address: make that first call
 * before any stream capture.  All calls share the array: calls that overlap on
 * the GPU race.  Synchronises `stream`; results in out[0..n_masks). */
int z2_zsums_static(int32_t n_qubits, int32_t precision, const void *state, const uint64_t *masks, int32_t n_masks,
                    double *out, void *stream);

/* ---- batched runs: a lambda sweep (many independent adiabatic runs) ------- */
typedef struct {
    int32_t d, L[3];      /* lattice                                  */
    z2_run_params params; /* schedule, decomposition, precision       */
} z2_run_spec;

#define Z2_SWEEP_PLAIN 0   /* one run after another on one stream, each synchronised            */
#define Z2_SWEEP_STREAMS 1 /* runs spread over n_streams streams, all enqueued before one wait  */
#define Z2_SWEEP_GRAPHS 2  /* as STREAMS, each run (|+>, M steps, observables) one CUDA graph   */
#define Z2_SWEEP_PERSISTENT 3 /* every complex64 run of 14 to 21 qubits evolved in one persistent
                                 launch (gangs of co-resident CTAs take runs from a device queue);
                                 observables and the other runs follow on n_streams streams
                                 (runs of 22 or more qubits fill the GPU with their own plans) */

/* Runs specs[0 .. n) (each: |+>^N, M steps, observables at s = 1, no
 * fidelity) and writes out[i]; out[i].status is that run's status.  The
 * library allocates and frees the device states (n_streams of the largest
 * size; all states at once in PERSISTENT mode).  Returns Z2_OK if every run
 * succeeded, else the first error.  The
 * result of a run does not depend on the mode or on the other runs (the same
 * kernels run on the same data in the same order). */
int z2_sweep(z2_ctx *ctx, const z2_run_spec *specs, int32_t n, int32_t mode, int32_t n_streams, z2_results *out);

/* ---- serving: a request loop with continuous batching --------------------
 * A server owns a worker thread that admits submitted runs in arrival order
 * (within the size classes of z2_server_set_option) as soon as a run slot is
 * free and the run's device memory (its state) fits the HBM budget, starts
 * each on its own stream (so
 * runs that arrive while others are on the GPU overlap with them), keeps its
 * state resident until it finishes, then returns the memory.  A run's result
 * does not depend on what else is running.  While a server exists its
 * context must not be used by other calls; all server calls are thread-safe. */
typedef struct {
    uint64_t submitted, completed, rejected, cancelled;
    int32_t active;           /* runs currently on the GPU            */
    int32_t queued;           /* runs waiting for admission           */
    size_t hbm_in_use;        /* bytes held by active runs            */
    size_t hbm_peak;          /* largest hbm_in_use so far            */
} z2_serve_stats;

/* hbm_budget: device bytes the server may hold for run states (0 = 80% of
 * the free memory); max_slots: most runs on the GPU at once (1..64). */
int z2_server_create(z2_ctx *ctx, size_t hbm_budget, int32_t max_slots, z2_server **out);
/* Admission by size class.  A run of at least Z2_SERVE_OPT_LARGE_QUBITS
 * qubits (default 22) fills every SM with each of its pass kernels, so
 * running several such runs at once only interleaves them; at most
 * Z2_SERVE_OPT_MAX_LARGE of them (default 2) are admitted at a time.  Smaller
 * runs take any free slot beside them, passing a large run that waits only for
 * a large-run place (it keeps its place in the queue).  The HBM budget still
 * admits in arrival order.  Z2_ERR_ARG for values out of range (large_qubits
 * 1..35, max_large 1..64) or for changing the class size while runs are active. */
#define Z2_SERVE_OPT_LARGE_QUBITS 0
#define Z2_SERVE_OPT_MAX_LARGE 1
int z2_server_set_option(z2_server *srv, int32_t option, int32_t value);
/* Queue a run; *ticket identifies it.  Z2_ERR_BUDGET if it can never fit. */
int z2_server_submit(z2_server *srv, const z2_run_spec *spec, uint64_t *ticket);
/* *done = 1 once the run has finished (then *out holds its results, with
 * out->status its status) or was cancelled; 0 while queued or running. */
int z2_server_poll(z2_server *srv, uint64_t ticket, int32_t *done, z2_results *out);
/* Block until the run has finished (or timeout_s seconds, < 0 = forever);
 * Z2_ERR_DEVICE_TIMEOUT if the wait ran out. */
int z2_server_wait(z2_server *srv, uint64_t ticket, double timeout_s, z2_results *out);
/* Cancel a queued run (a running one finishes normally). */
int z2_server_cancel(z2_server *srv, uint64_t ticket);
int z2_server_stats(z2_server *srv, z2_serve_stats *out);
/* Seconds a finished run waited for admission and spent running (host
 * monotonic clock, submit -> admission -> completion seen by the worker). */
int z2_server_request_times(z2_server *srv, uint64_t ticket, double *queued_s, double *run_s);
/* Device-clock timestamps of a finished run, in seconds since the server was
 * created (CUDA events on the run's stream): *first_s once its first kernel
 * (the |+> initialisation) has run, *end_s once its last work has.  Two runs
 * whose intervals intersect had work on the GPU at the same time. */
int z2_server_request_device_times(z2_server *srv, uint64_t ticket, double *first_s, double *end_s);
/* Stop the worker after the runs already admitted finish; queued runs are
 * cancelled; frees everything. */
int z2_server_destroy(z2_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* Z2LGT_H */
