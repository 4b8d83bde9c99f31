/*
 * sq.h -- C ABI of the GB300-native asqtad staggered CG library.
 *
 * The library solves (m^2 - D_eo D_oe) x = b on the even sites of a 4-d
 * lattice, where D is the asqtad (improved staggered) Dirac operator with
 * fat one-hop links F and long three-hop (Naik) links L:
 *
 *   (D psi)(x) = 1/2 sum_mu eta_mu(x) [ F_mu(x) psi(x+mu) - F_mu(x-mu)^dag psi(x-mu)
 *                                      + L_mu(x) psi(x+3mu) - L_mu(x-3mu)^dag psi(x-3mu) ]
 *
 * with eta_0 = 1, eta_1 = (-1)^x, eta_2 = (-1)^(x+y), eta_3 = (-1)^(x+y+z).
 * This is the mixed-precision CG inverter for asqtad quarks that the paper
 * ("Code Optimization on Kepler GPUs and Xeon Phi", Sec. 2, Fig. 1 and
 * Table 2; Sec. 3, Table 4) times on a 20^3 x 64 lattice, and the entry
 * points play the part of the application-to-solver interface of Sec. 3
 * (the staggered-CG call the authors added between CPS and QUDA).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * dims      int[4] = {Lx, Ly, Lz, Lt}; every extent even and >= 2; V = product,
 *           Vh = V/2.
 * site_lex  x + Lx*(y + Ly*(z + Lz*t)).
 * links     host/device array [site_lex][mu][row][col] of complex128
 *           (interleaved re, im), mu = 0..3 for x, y, z, t; 4*9*V complex.
 *           Fat links carry c1 and long links carry c3 (no coefficient is
 *           applied inside the library).
 * vectors   parity-half colour vectors in "canonical" layout: [i][colour]
 *           complex128, i = site_lex / 2 ranking the parity's sites; 3*Vh
 *           complex.  Solves act on the even parity.
 * packed    the library's device layout for one parity-half vector, used by
 *           dslash_apply and mdagm_apply (see sq_spinor_bytes):
 *             SQ_PREC_F64: 3 planes of double2 (colour c at plane c);
 *             SQ_PREC_F32: a float4 plane (c0.re, c0.im, c1.re, c1.im) then a
 *                          float2 plane (c2.re, c2.im);
 *             SQ_PREC_I16: one 16-byte record per site: three 32-bit words
 *                          holding the colour's (re, im) 16-bit codes (re in
 *                          the low half) as excess-32768 integers, then the
 *                          site norm n as an FP32; value = code * n / 32767.
 *           A plane holds `stride` sites (Vh rounded up to a multiple of 64).
 * streams   `void *stream` is a cudaStream_t.  The blocking calls (solves,
 *           dirac_apply) run on it, or on the context's stream when it is
 *           NULL or a default stream, after waiting for that stream's work.
 *           The asynchronous calls (dslash_apply, dslash_apply_multi,
 *           mdagm_apply, mdagm_apply_static, the pack helpers,
 *           gauge_fatten*, npr_four_fermion) run on `stream` as given: NULL
 *           is the legacy default stream, as in CUDA, so they are ordered
 *           with all other work on it (torch's default stream included).
 * errors    every call returns an sq_status; nothing aborts or throws.
 *           Non-finite inputs give SQ_ERR_NONFINITE.
 * ownership the caller owns every pointer it passes; calls that take host
 *           data copy it before returning.  The library owns the device
 *           memory behind contexts and gauge ids.
 */
#ifndef SQ_H
#define SQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sq_ctx sq_ctx;

typedef enum {
    SQ_OK = 0,
    SQ_PENDING = 1,          /* serve_poll: not finished within the timeout     */
    SQ_NOT_CONVERGED = 2,    /* max_iter reached; x and stats are still written */
    SQ_ERR_ARG = -1,
    SQ_ERR_OOM = -2,         /* device allocation or the HBM budget refused     */
    SQ_ERR_CUDA = -3,
    SQ_ERR_NONFINITE = -4,
    SQ_ERR_TIMEOUT = -5,
    SQ_ERR_BUSY = -6,
    SQ_ERR_NOTFOUND = -7,
    SQ_ERR_UNSUPPORTED = -8  /* e.g. 12-real long links on links that are not c*SU(3) */
} sq_status;

typedef enum { SQ_PREC_F64 = 0, SQ_PREC_F32 = 1, SQ_PREC_I16 = 2 } sq_prec;

/* gauge_load flags */
#define SQ_GAUGE_DEVICE_PTRS    0x1u  /* fat/lng are device pointers              */
#define SQ_GAUGE_ANTIPERIODIC_T 0x2u  /* hops that wrap around t pick up -1        */
#define SQ_GAUGE_NO_F32         0x10u /* skip the FP32 forms                      */
#define SQ_GAUGE_NO_I16         0x20u /* skip the 16-bit forms                    */
#define SQ_GAUGE_NO_LONG12      0x40u /* skip the 12-real long-link forms         */
#define SQ_GAUGE_NO_F64         0x80u /* skip the FP64 forms (no solves then)     */

/* sq_cg_opts.flags */
#define SQ_CG_DEVICE_PTRS   0x1u  /* src/x are device pointers (canonical layout) */
#define SQ_CG_INITIAL_GUESS 0x2u  /* x holds the starting guess on input          */
#define SQ_CG_NO_GRAPH      0x4u  /* launch kernels directly, no CUDA graph       */

typedef struct {
    int precision;     /* sloppy precision: SQ_PREC_F64 = plain FP64 CG (default F32) */
    int long_recon;    /* 18 or 12: long links stored 18-real or 12-real (default 18) */
    double delta;      /* reliable update when |r| < delta * max|r| since the last
                          one; < 0 (default): 0.001 for FP32, 0.1 for 16-bit sloppy
                          vectors; ignored for plain FP64 CG                         */
    int max_iter;      /* default 100000                                              */
    int block_iters;   /* CG iterations per graph launch (default 16)                 */
    unsigned flags;    /* SQ_CG_* */
    void *stream;      /* cudaStream_t the solve runs on (it still returns only when
                          done); NULL or a default stream: the context's stream,
                          after the work already queued on that default stream  */
} sq_cg_opts;

typedef struct {
    int status;            /* sq_status of this solve                          */
    int iterations;
    int reliable_updates;  /* FP64 true-residual recomputations                */
    double true_residual;  /* |b - A x| / |b|, FP64, computed on the GPU       */
    double seconds;        /* wall time of the solve (host clock)              */
    double gflops;         /* 2364 flop per even site per iteration            */
    /* Launch shapes of the CG's two sloppy Dslash kernels as launched (the
     * tuner's choice, or a SQ_TUNE_CACHE entry): threads per block and
     * right-hand sides per thread of the D_oe kernel (with the reduction)
     * and of the D_eo kernel (with the update).  0 where no batched CG ran. */
    int oe_block, oe_rhs_tile, eo_block, eo_rhs_tile;
} sq_cg_stats;

typedef struct {
    uint64_t submitted, completed, rejected;
    int queued, running;
    double p50_ms, p99_ms, mean_ms;   /* submit -> result ready, completed requests */
    double solves_per_s;              /* completed / (last completion - first submit) */
    size_t hbm_in_use, hbm_budget;
} sq_serve_stats;

/* ---- context -------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may hold (gauge fields + solver and serving workspaces;
 * not the transient staging of gauge_load); 0 = 90% of the device's free
 * memory.  Returns SQ_ERR_CUDA without a usable device. */
int sq_create(sq_ctx **out, int device, size_t hbm_budget_bytes);
int sq_destroy(sq_ctx *ctx);
const char *sq_strerror(int status);
void sq_cg_opts_default(sq_cg_opts *opts);

/* Number of kernel launches the context has issued (graph launches count each
 * kernel node), for launch accounting. */
uint64_t sq_kernel_launches(const sq_ctx *ctx);

/* ---- gauge field ---------------------------------------------------------- */

/* Load fat and long links (layout above) and pack them into the device forms
 * used by the Dslash: for each output parity, per site, the 16 hop matrices
 * F_mu(x), F_mu(x-mu)^dag, L_mu(x), L_mu(x-3mu)^dag, stored site-major in
 * 16-byte planes, in FP64, FP32 and 16-bit (global scale per link kind), with
 * the long links also in 12-real form (third row rebuilt as
 * conj(row0 x row1)/s, s the common scale of the long links, found from
 * det L = s^3 and checked on every link).  One-time; the caller may free the
 * inputs on return.  The paper's links come from the MILC asqtad ensemble
 * (Sec. 2, Fig. 1); any fat/long pair in this layout is accepted. */
int gauge_load(sq_ctx *ctx, const int dims[4], const double *fat, const double *lng,
               unsigned flags, int *gauge_id);
int gauge_free(sq_ctx *ctx, int gauge_id);

/* Fat and long links from thin links, on the device in FP64:
 *   F_mu(x) = c1 [ U_mu(x) + w sum_{nu != mu} ( U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
 *              + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ) ] / (1 + 6w),
 *   L_mu(x) = c3 U_mu(x) U_mu(x+mu) U_mu(x+2mu),
 * with periodic neighbours (w = staple_weight; the benchmark workloads use
 * c1 = 9/8, c3 = -1/24, w = 0.1).  This stands in for the asqtad link
 * fattening that produces the paper's MILC links (Sec. 2, Fig. 1); it is not
 * MILC's full path set.  thin_dev, fat_dev, lng_dev: distinct device arrays
 * in the links layout above.  Asynchronous on `stream`; NULL means the legacy
 * default stream (ordered with all other work on it). */
int gauge_fatten(sq_ctx *ctx, const int dims[4], const double *thin_dev, double c1, double c3,
                 double staple_weight, double *fat_dev, double *lng_dev, void *stream);

/* The asqtad action's fat and Naik links from thin links, on the device in
 * FP64: MILC's path set for the fat link -- the one-link term, the 6
 * three-link, 24 five-link and 48 seven-link staples and the 6 Lepage terms
 * of direction mu, each the product of links along its path -- and the Naik
 * link c_N U_mu(x) U_mu(x+mu) U_mu(x+2mu).  coeffs = {one-link, 3-staple,
 * 5-staple, 7-staple, Lepage, Naik}; with the paths oriented as
 *   (s nu) mu (-s nu),  (r rho)(s nu) mu (-s nu)(-r rho),  ...,
 *   (s nu)(s nu) mu (-s nu)(-s nu)
 * (a hop +d at y multiplies by U_d(y), a hop -d by U_d(y-d)^dag), the
 * tree-level asqtad values are {5/8, 1/16, 1/64, 1/384, -1/16, -1/24}, which
 * give 9/8 and -1/24 on unit links.  The paper's lattices are MILC asqtad
 * ensembles (Sec. 2, Fig. 1).  Arrays and `stream` as for gauge_fatten; the
 * paths are built as nested staple fields in a stream-ordered device scratch
 * of 288 bytes per site, taken and returned on `stream` (outside the HBM
 * budget). */
int gauge_fatten_asqtad(sq_ctx *ctx, const int dims[4], const double *thin_dev,
                        const double coeffs[6], double *fat_dev, double *lng_dev, void *stream);

/* gauge_fatten followed by gauge_load (the smeared links of the paper's MILC
 * lattices, Sec. 2, built here from thin links): thin links in (host
 * pointer, or device with SQ_GAUGE_DEVICE_PTRS), a gauge id out.  The fat and long links exist
 * on the device only transiently (staging outside the HBM budget, freed on
 * return).  Other flags as for gauge_load. */
int gauge_load_thin(sq_ctx *ctx, const int dims[4], const double *thin, double c1, double c3,
                    double staple_weight, unsigned flags, int *gauge_id);

/* Solve M x = b on the whole lattice, M = m + D, by BiCGstab (van der Vorst,
 * SIAM J. Sci. Stat. Comput. 13 (1992) 631) applied to M itself -- the
 * BiCG-family inverter the paper lists beside CG among QUDA's (Sec. 3) -- in
 * FP64 on the device.  The recursion stops when |r| / |b| <= tol; the FP64
 * residual b - M x is then recomputed, and the solve restarts from it (a new
 * shadow residual) unless it is <= tol too; it also restarts on a breakdown
 * (rho = 0 or <r^, v> = 0), at most 64 times in all (then SQ_NOT_CONVERGED).  stats->iterations counts BiCGstab
 * steps (two M products each), stats->reliable_updates the recomputed
 * residuals, stats->true_residual the last of them.  M is not Hermitian, and
 * on staggered spectra (m + i lambda) BiCGstab needs many more products than
 * the even-odd CG of cg_solve_full; it is here for comparison.
 * opts->precision: SQ_PREC_F64 runs everything in FP64; SQ_PREC_F32 (the
 * sq_cg_opts default) keeps the vectors and the Dslash in FP32 and folds the
 * FP32 solution increment into an FP64 solution at reliable updates, when
 * |r| < delta max|r| since the last one (opts->delta, < 0: 0.1) or the
 * recursion claims convergence; r is then the FP64 residual b - M x.  NULL
 * opts: FP64.  Arrays, flags (SQ_CG_DEVICE_PTRS, SQ_CG_INITIAL_GUESS),
 * max_iter and stream as cg_solve_full; SQ_ERR_UNSUPPORTED for 16-bit or for
 * a field without the FP64 (and, for FP32, FP32) 18-real links. */
int bicgstab_solve_full(sq_ctx *ctx, int gauge_id, const double *src, double mass, double tol,
                        const sq_cg_opts *opts, double *x, sq_cg_stats *stats);

/* ---- NPR four-fermion operator (Sec. 2, Eq. 1, Fig. 2, Table 3) ---------- */

#define SQ_NPR_MAX_OPS 16  /* operators per kernel launch */

/* The hypercube spin-taste matrix of Eq. 1,
 *   (gamma_S x xi_F)_{AB} = Tr(gamma_A^dag gamma_S gamma_B gamma_F^dag) / 4,
 * gamma_X = gamma_1^{X_0} gamma_2^{X_1} gamma_3^{X_2} gamma_4^{X_3} (Euclidean),
 * in the form the GPU uses: row A has one nonzero entry, sign[A] (+1 or -1)
 * at column partner[A] = A ^ S ^ F.  S, F, A: 4-bit masks, bit mu for
 * direction mu = x, y, z, t.  Host only (no device work); SQ_ERR_ARG for a
 * mask outside 0..15 or a null array. */
int sq_spin_taste(int s, int f, int partner[16], int sign[16]);

/* The one-colour four-fermion operator of the paper's NPR code, Eq. 1, in
 * FP64 on the device, for nops operators (S1, F1, S2, F2) (4-bit masks, host
 * array ops[nops][4], 0 <= nops <= 2^20; they are processed SQ_NPR_MAX_OPS at
 * a time, each group recomputing the averaged links and sandwiches -- about
 * a sixth of a group's work at 8 operators, less at 16):
 *   O[a1][a2][a3][a4](z) = sum_{A,B,C,D} sum_{c1..c4}
 *       conj(G1(z_A)[c1][a1]) (gamma_S1 x xi_F1)_{AB} G2(z_B)[c2][a2]
 *     * conj(G3(z_C)[c3][a3]) (gamma_S2 x xi_F2)_{CD} G4(z_D)[c4][a4]
 *     * U_AD(z)[c1][c4] U_CB(z)[c3][c2]
 * over the hypercubes z (0 <= z_mu < L_mu / 2) with corner sites
 * z_A = 2z + A.  U_AD(z) is the mean of the link products over the shortest
 * paths from z_A to z_D inside the hypercube (a step +mu from y is U_mu(y), a
 * step -mu is U_mu(y-mu)^dag).  The quark fields are the source-colour
 * columns a of the propagators G^f, the antiquark fields (flavours 1, 3)
 * their complex conjugates.
 *   links_dev   device, [site_lex][mu][3][3] complex128 (any links: thin or
 *               smeared);
 *   props_dev   four device arrays, [site_lex][colour][source colour]
 *               complex128;
 *   out_dev     device, [op][a1][a2][a3][a4] complex128: the sum over z;
 *   out_hc_dev  NULL, or device [z][op][a1][a2][a3][a4] complex128 with
 *               z = z_x + Hx (z_y + Hy (z_z + Hz z_t)), H = L / 2.
 * Device arrays 16-byte aligned; all extents even.  Asynchronous on `stream`,
 * NULL meaning the legacy default stream (a stream-ordered scratch of
 * 16 * 81 * nops bytes per CTA is taken and returned on it).  The sum over z
 * is deterministic.  The inputs are not checked for finiteness. */
int npr_four_fermion(sq_ctx *ctx, const int dims[4], const double *links_dev,
                     const double *const props_dev[4], int nops, const int *ops,
                     double *out_dev, double *out_hc_dev, void *stream);

/* Bytes of one packed parity-half vector of `prec` for this gauge field's
 * lattice, and the plane stride in sites (the device layout of this library;
 * the paper prints none). */
int sq_spinor_bytes(sq_ctx *ctx, int gauge_id, int prec, size_t *bytes, int *stride);

/* Canonical (complex128) <-> packed device vector of one parity (this
 * library's layout; the paper prints none).  Both pointers are device
 * pointers; asynchronous on `stream`. */
int sq_pack_spinor(sq_ctx *ctx, int gauge_id, int prec, const double *canon_dev,
                   void *packed_dev, void *stream);
int sq_unpack_spinor(sq_ctx *ctx, int gauge_id, int prec, const void *packed_dev,
                     double *canon_dev, void *stream);

/* ---- operators ------------------------------------------------------------ */

/* out = D_{p,1-p} in: the asqtad Dslash from parity 1-out_parity to parity
 * out_parity (the 16 SU(3) mat-vecs per site above; the operator in which the
 * paper's CG inverter spends its time, Sec. 2, Fig. 1), in `prec` with long
 * links in `long_recon` (18 or 12) form.  in/out are packed device vectors
 * (distinct buffers).  Asynchronous on `stream`; no host synchronisation. */
int dslash_apply(sq_ctx *ctx, int gauge_id, int out_parity, int prec, int long_recon,
                 const void *in_dev, void *out_dev, void *stream);

/* out_j = D_{p,1-p} in_j for nrhs right-hand sides in one launch (1 <= nrhs
 * <= 64): the Dslash of dslash_apply, with each link read once for a tile of
 * right-hand sides per thread (the batched form of the operator the paper's
 * CG spends its time in, Sec. 2; batching is this library's).  in/out:
 * nrhs packed vectors back to back, each sq_spinor_bytes long, in distinct
 * buffers.  The tile and block size are the tuner's (sq_tuned_launch, mode
 * 0).  Asynchronous on `stream`. */
int dslash_apply_multi(sq_ctx *ctx, int gauge_id, int out_parity, int prec, int long_recon,
                       int nrhs, const void *in_dev, void *out_dev, void *stream);

/* The launch shape the library uses for one of its Dslash kernels on this
 * gauge field: threads per block and right-hand sides per thread, for `nrhs`
 * systems in `prec` with `long_recon`-real long links.  mode: 0 the plain
 * Dslash (dslash_apply, dslash_apply_multi, the FP64 reliable-update pair),
 * 1 with the m^2 epilogue (mdagm_apply, multi-shift), 3 the CG's D_oe kernel
 * with its reduction, 4 the CG's D_eo kernel with its update.  The shape is
 * chosen by timing the candidates on first use (which allocates scratch and
 * synchronises `stream`) unless SQ_TUNE_CACHE or an earlier call fixed it;
 * for modes 1, 3 and 4, which run in chains of dependent launches, the
 * smallest block within 3 % of the fastest is taken.
 * (The paper's QUDA path tunes its launches at run time, Sec. 3.) */
int sq_tuned_launch(sq_ctx *ctx, int gauge_id, int prec, int long_recon, int nrhs, int mode,
                    void *stream, int *block, int *rhs_tile);

/* Device time of one of those Dslash kernels (modes as sq_tuned_launch) at
 * the launch shape the library uses: `reps` back-to-back launches on
 * synthetic vectors (the gauge field's own links, running systems for the
 * reducing modes), timed with CUDA events on `stream` after a warm-up;
 * *us_per_launch is the mean.  For rooflines of the kernels the solvers run
 * inside CUDA graphs (the paper measures its CG in GFLOPS, Table 2).
 * Allocates scratch for the call and synchronises `stream`. */
int sq_time_dslash(sq_ctx *ctx, int gauge_id, int prec, int long_recon, int nrhs, int mode,
                   int reps, void *stream, float *us_per_launch);

/* out = (m^2 - D_eo D_oe) in on the even parity: the operator of the paper's
 * even-odd CG inverter (Sec. 2), as two Dslash kernels (the second with the
 * m^2 epilogue).  Uses a
 * context-owned odd-parity temporary. */
int mdagm_apply(sq_ctx *ctx, int gauge_id, int prec, int long_recon, double mass,
                const void *in_dev, void *out_dev, void *stream);

/* Same operator as mdagm_apply, for callers that cannot let the library
 * allocate device memory when they call it: applications that reserve all of
 * HBM up front through their own allocator or memory pool and forbid
 * libraries to allocate behind it, and latency-critical loops in which a
 * first-use cudaMalloc would be an unpredictable stall (mdagm_apply
 * allocates its temporary on first use per gauge field and precision).  (The
 * paper has no counterpart; this is an interface of this library only.)
 * The odd-parity temporary lives in one fixed device array of
 * SQ_STATIC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits; the call allocates nothing (no cudaMalloc, no cudaFree, no
 * tuning).  The packed vector of one parity (sq_spinor_bytes) must fit that
 * array -- e.g. up to 524288 sites per parity in FP32 (a 20^3 x 64 lattice
 * has 256000) -- otherwise SQ_ERR_ARG.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) as a one-time set-up;
 * make that first call before any stream capture.  All calls share the array
 * and it keeps the last call's contents; the temporary is fully rewritten by
 * each call before it is read, so nothing needs clearing, but calls that
 * overlap on the GPU (other streams, other threads) race on it: serialise
 * them.  in/out and stream as for mdagm_apply. */
#define SQ_STATIC_SCRATCH_BYTES (12u << 20)
int mdagm_apply_static(sq_ctx *ctx, int gauge_id, int prec, int long_recon, double mass,
                       const void *in_dev, void *out_dev, void *stream);

/* ---- solvers -------------------------------------------------------------- */

/* Solve (m^2 - D_eo D_oe) x = b to |b - A x| / |b| <= tol: CG in the sloppy
 * precision opts->precision with FP64 reliable updates (the FP64 true
 * residual is recomputed, and CG restarted from it, whenever |r| falls below
 * delta times its maximum since the previous update, and before returning);
 * the solution accumulates in FP64.  With precision SQ_PREC_F64 it is plain
 * FP64 CG.  This is the paper's mixed-precision CG (Sec. 2: "most of the
 * calculations are performed in single precision"; Sec. 3).  src/x are
 * canonical even-parity vectors, host pointers unless SQ_CG_DEVICE_PTRS.
 * opts may be NULL (defaults).  stats may be NULL. */
int cg_solve(sq_ctx *ctx, int gauge_id, const double *src_even, double mass, double tol,
             const sq_cg_opts *opts, double *x_even, sq_cg_stats *stats);

/* Batched solve of nrhs systems (m_j^2 - D_eo D_oe) x_j = b_j on one gauge
 * field, each by the CG of cg_solve (the paper's inverter, Sec. 2, solves one
 * system at a time; batching is this library's): every Dslash streams each
 * link once for all right-hand sides.
 * src/x: nrhs canonical vectors back to back; masses: nrhs values; stats:
 * nrhs entries (may be NULL).  Each system follows cg_solve's algorithm and
 * stops on its own. */
int cg_solve_multi(sq_ctx *ctx, int gauge_id, int nrhs, const double *src,
                   const double *masses, double tol, const sq_cg_opts *opts,
                   double *x, sq_cg_stats *stats);

/* Multi-shift CG (not in the paper; the masses of Sec. 2's inverter solved
 * together): (m_i^2 - D_eo D_oe) x_i = b for nshift masses from one Krylov
 * space (Jegerlehner's shifted recurrences, hep-lat/9612014), run in the sloppy
 * precision to max(tol, 1e-6 for FP32 / 1e-3 for 16-bit), then refined per
 * shift by the batched mixed-precision CG above started from the shifted
 * solutions.  x: nshift canonical vectors; stats: nshift entries (may be NULL). */
int cg_solve_multishift(sq_ctx *ctx, int gauge_id, const double *src, int nshift,
                        const double *masses, double tol, const sq_cg_opts *opts,
                        double *x, sq_cg_stats *stats);

/* Solve M x = b on the whole lattice, M = m + D on both parities (D as
 * above).  Staggered D only joins sites of opposite parity, so M x = b splits
 * into the even-site system of cg_solve and a direct odd-site step:
 *   (m^2 - D_eo D_oe) x_e = m b_e - D_eo b_o     (CG as in cg_solve, with opts),
 *   x_o = (b_o - D_oe x_e) / m.
 * For the even residual r_e of that system, b - M x = (r_e / m, 0), so the
 * even system is solved to tol * m |b| / |m b_e - D_eo b_o|, which makes
 * |b - M x| / |b| <= tol.  stats->true_residual is that full-lattice FP64
 * residual, recomputed on the device from x after the solve (iterations and
 * reliable updates are the even solve's).  src/x: full-lattice vectors
 * [site_lex][colour] complex128 (3 V complex), host pointers unless
 * SQ_CG_DEVICE_PTRS; with SQ_CG_INITIAL_GUESS the even sites of x start the
 * CG.  Device scratch for the call is taken from the HBM budget and released
 * on return.  This is the staggered equation the paper's CG inverter solves
 * (Sec. 2, Fig. 1). */
int cg_solve_full(sq_ctx *ctx, int gauge_id, const double *src, double mass, double tol,
                  const sq_cg_opts *opts, double *x, sq_cg_stats *stats);

/* out = (m + D) in on the whole lattice, in FP64: the staggered matrix of the
 * paper's inverter (Sec. 2) without even-odd preconditioning.  in_dev/out_dev: distinct device
 * full-lattice vectors [site_lex][colour] complex128.  Uses device scratch
 * for the call (HBM budget) and returns once out is written. */
int dirac_apply(sq_ctx *ctx, int gauge_id, double mass, const double *in_dev, double *out_dev,
                void *stream);

/* ---- serving -------------------------------------------------------------- */

/* Continuous-batching request loop (not in the paper: a serving interface of
 * this library around the solves of Sec. 2).  serve_submit copies the host
 * source and queues one solve; a scheduler thread admits queued requests into free slots
 * of the running batched CG of their gauge field (at iteration-block
 * boundaries) while the HBM budget allows, runs the batches of all gauge
 * fields concurrently on separate streams and retires converged slots.
 * Options of a served solve: sq_cg_opts defaults (FP32 sloppy, 18-real). */
int serve_submit(sq_ctx *ctx, int gauge_id, const double *src_even, double mass, double tol,
                 uint64_t *ticket);

/* Wait up to timeout_us (0: do not wait; <0: forever) for a ticket; on
 * completion copy x into x_even (host, may be NULL) and stats, release the
 * ticket and return the solve's status.  SQ_PENDING if not yet done;
 * SQ_ERR_NOTFOUND for an unknown or already released ticket. */
int serve_poll(sq_ctx *ctx, uint64_t ticket, double *x_even, sq_cg_stats *stats,
               int timeout_us);

/* Cancel a queued or running request (its ticket then polls SQ_ERR_NOTFOUND). */
int serve_cancel(sq_ctx *ctx, uint64_t ticket);

/* Serving counters and latency percentiles since the context was created (or
 * the last reset). */
int serve_stats(sq_ctx *ctx, sq_serve_stats *stats, int reset);

/* Slots per gauge-field batch (default 8, at most 16); set before submitting. */
int serve_configure(sq_ctx *ctx, int slots_per_batch, int block_iters);

#ifdef __cplusplus
}
#endif

#endif /* SQ_H */
