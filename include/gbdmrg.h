/*
 * gbdmrg.h -- C ABI of a single-GPU (GB300, sm_103a) two-site DMRG hot path:
 * block-sparse effective-Hamiltonian products inside Davidson, truncation,
 * renormalisation, sweeps, and the parallel pack/unpack (serialise /
 * deserialise) of block-sparse environments with host offload.
 *
 * Method: arXiv:2412.04676.  Eq. 1 (Hamiltonian), Eq. 2 (MPS), Eq. 3
 * (variational minimum), Sec. II.B (two-site step: pre-processing,
 * diagonalisation, post-processing; Fig. 3a), Sec. III.A (asynchronous save),
 * Sec. III.B.2 (exact-size parallel serialisation), Sec. III.B.3
 * (self-contained packages), Sec. III.B.4 (load-after-renormalise ordering).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Orbitals (sites) 0..L-1.  Local basis per orbital: 0=|0>, 1=|up>, 2=|dn>,
 * 3=|updn> = c+_up c+_dn |0>.  Quantum numbers q = (n, tsz), tsz = twice S_z,
 * counted from the left: bond (cut) k carries those of orbitals 0..k-1.
 * The two-site step at site b works on orbitals (b, b+1); its enlarged left
 * block is (cut-b block + orbital b), its enlarged right block is
 * (orbital b+1 + cut-(b+2) block).
 *
 * Wavefunction layout ("sector-major"): sectors Q of the enlarged left block
 * that also exist on the enlarged right block, in ascending (n, tsz)
 * lexicographic order; each sector is a row-major dense matrix
 * rows = dim of the enlarged left block in Q, cols = dim of the enlarged
 * right block in Q.  Rows list the local states s = 0..3 in order, each
 * followed by the states of cut-b sector Q - q_s; columns list s = 0..3 in
 * order, each followed by the states of cut-(b+2) sector Q + q_s.
 *
 * Status: every call returns int: 0 = OK, < 0 = error, > 0 = warning.
 * gbd_last_error() gives the message of the last failed call made by the
 * calling thread, whatever context it was made on; it takes no context
 * because some failures (gbd_create, gbd_pack_noalloc) have none.  No
 * exception crosses the ABI and no device code traps.
 *
 * Ownership: the library owns all device memory and pinned host memory it
 * allocates; callers own every array they pass in, which is copied (or fully
 * consumed) before the call returns unless a comment says otherwise.
 * Device pointers passed in must stay valid for the duration of the call.
 */
#ifndef GBDMRG_H
#define GBDMRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    GBD_OK = 0,
    GBD_ERR_ARG = -1,          /* bad argument, size or state of inputs         */
    GBD_ERR_DEVICE_OOM = -2,   /* cudaMalloc failed                              */
    GBD_ERR_HOST_OOM = -3,     /* pinned host allocation failed                  */
    GBD_ERR_CUDA = -4,         /* any other CUDA / cuSOLVER error                */
    GBD_ERR_TIMEOUT = -5,      /* a bounded wait on an IO event ran out          */
    GBD_ERR_CORRUPT = -6,      /* package magic / checksum / metadata mismatch   */
    GBD_ERR_STATE = -7,        /* call out of order (e.g. no integrals loaded)   */
    GBD_WARN_NOT_CONVERGED = 1, /* Davidson hit its product limit                */
    GBD_WARN_PRECISION_FLOOR = 2 /* mixed Davidson: its anchors stopped above
                                    dav_tol (an anchor that did not cut the
                                    best exact residual by a fifth, or GBD_MAX_ANCHORS of
                                    them: the floor the BF16x3 products leave);
                                    the result is the anchored pair with the
                                    smallest exact residual                    */
};

/* Most accurate anchor products of one mixed Davidson solve. */
#define GBD_MAX_ANCHORS 6

/* H_eff product forms.  GBD_FP64: FP64 GEMMs.  GBD_MIXED_BF16X3: every
 * operand split elementwise into BF16 hi + lo, products hh + hl + lh on the
 * tensor cores with FP32 accumulation (~1e-5 relative).  GBD_SLICED_BF16:
 * every operand row cut into 64-wide blocks, each written exactly as four
 * BF16 slices on the power-of-two grid of the block maximum (the error-free
 * splitting of Ozaki et al.); the ten slice products of orders <= 4 run on the
 * tensor cores, the two leading orders accumulating exactly in FP32 (about
 * 2^-30 relative to the row maxima).  GBD_SLICED_BF16 is a product form for
 * gbd_apply_heff and for Davidson anchors (mixed_polish = 2), not a
 * context precision. */
enum { GBD_FP64 = 0, GBD_MIXED_BF16X3 = 1, GBD_SLICED_BF16 = 2, GBD_FP64_PER_BLOCK = 3, GBD_BF16X3_TWO_PHASE = 4,
       GBD_BF16X3_FUSED = 5 };
/* GBD_FP64_PER_BLOCK: the FP64 product with one kernel launch per sector
 * block GEMM task instead of one grouped launch per phase (same kernel, same
 * tiles, bitwise the same result); a comparison form for gbd_apply_heff.
 * GBD_BF16X3_TWO_PHASE / GBD_BF16X3_FUSED: the BF16x3 product in two
 * kernels with X stored in HBM between them / in the fused kernel, whatever
 * gbd_config.bf16x3_fused says (same split products, another summation
 * order); comparison forms for gbd_apply_heff. */

typedef struct gbd_ctx gbd_ctx;

typedef struct {
    int L;              /* orbitals                                             */
    int N;              /* electrons                                            */
    int tsz;            /* twice S_z                                            */
    int D;              /* maximum kept states per bond (truncation)            */
    int precision;      /* GBD_FP64 or GBD_MIXED_BF16X3 (H_eff products only)   */
    double dav_tol;     /* Davidson residual norm tolerance (FP64 norm); mixed
                           precision stops at max(dav_tol, 2e-5) or when the
                           residual stalls at the rounding floor of its
                           products (< 10% gain over 8 iterations)           */
    int dav_max_sub;    /* Davidson subspace size before restart                */
    int dav_keep;       /* Ritz vectors kept at restart                         */
    int dav_max_matvec; /* product limit -> GBD_WARN_NOT_CONVERGED              */
    int offload;        /* 1: environments are packed to pinned host RAM after
                           creation and unpacked on demand (Sec. III.A)       */
    int device;         /* CUDA device ordinal                                  */
    int switch_cut;     /* cut from which two-operator sets are stored as
                           complementary sums; 0 = automatic (L/2 - 1, so the
                           once-per-half-sweep switch transform is not at the
                           two central positions)                            */
    int io_timeout_ms;  /* bound on any host wait for an IO event              */
    unsigned long long seed; /* random initial MPS when none is imported       */
    int mixed_fp64_blocks; /* mixed products: 1 = the two block Hamiltonian
                              terms (H_left x 1, 1 x H_right) run in FP64
                              beside each BF16x3 product; 0 (default) = on
                              the tensor cores with the other terms        */
    int mixed_polish;   /* mixed Davidson anchors: at the tolerance or at the
                           rounding floor the Ritz vector gets an accurate
                           product; its Rayleigh quotient and residual decide
                           convergence, else the subspace restarts from it.
                           0: none (energy from mixed products), 1: FP64
                           products, 2 (default): GBD_SLICED_BF16 products;
                           with 2 the mixed form also runs the enlargement
                           and renormalisation GEMMs in the sliced form     */
    int fault_inject;   /* host-side fault injection for failure tests, 0 in
                           normal use; a sum of GBD_FAULT_* bits           */
    int autotune;       /* 1 (default): the BF16x3 phase-2 work-list shape is
                           chosen per position by timing candidate shapes on
                           its first products (gbd_tune_info); the choice is
                           cached under the position's sector-size histogram
                           and reused; 0: the fixed default shape          */
    int env_recompute;  /* with offload on: 0 (default) every environment is
                           saved to the pinned host store; k >= 2: only
                           environments at cuts divisible by k (and the two
                           chain ends) are saved, the others are dropped
                           after use and rebuilt when needed from the
                           nearest saved one towards their chain end, by
                           enlargement and renormalisation with the current
                           site isometries (recomputation instead of IO)  */
    long long host_store_bytes; /* with offload on: 0 (default) no bound on the
                           pinned host memory of saved environments; > 0: at
                           most this many bytes stay pinned, the least
                           recently used saved environments go to a spill
                           file (one per context, in $TMPDIR or /tmp,
                           removed with the process) through an IO thread
                           and are read back when a step needs them        */
    int low_memory;     /* mixed form with sliced anchors (mixed_polish = 2):
                           its products read only the tensor-core planes, so
                           the FP64 enlarged operators can be released once
                           both forms' planes are built (the diagonal first).
                           0 (default): only when the planes and the phase-1
                           buffer would not fit beside them; 1: always;
                           -1: never.  A later GBD_FP64 product at the same
                           position enlarges the operators again.          */
    int bf16x3_fused;   /* BF16x3 products: 0 (default) two kernels with X
                           stored in HBM between them; 1: one fused kernel
                           per product (each chunk of X = O^Lx psi is formed
                           in tensor memory, split into BF16 hi / lo there
                           and multiplied at once into the output tile, so X
                           never reaches HBM; half the DRAM traffic, but
                           slower on GB300: its chunk-by-chunk split is a
                           latency chain and its first MMAs are 64 wide)  */
} gbd_config;

/* Host-side fault injection (gbd_config.fault_inject).  Each failure is made
 * on the host; no device code is made to fault, trap or hang.
 *   GBD_FAULT_PINNED_ALLOC: every pinned host allocation of the offload
 *     store is refused -> GBD_ERR_HOST_OOM from the call that needed it.
 *   GBD_FAULT_IO_NEVER_READY: host waits on IO events never see them
 *     complete, so each runs out after io_timeout_ms -> GBD_ERR_TIMEOUT.
 *   GBD_FAULT_CORRUPT_HOST_COPY: before an offloaded environment is loaded
 *     back, one payload byte of its host copy is flipped -> the package
 *     checksum fails when the environment is first used (GBD_ERR_CORRUPT). */
enum { GBD_FAULT_PINNED_ALLOC = 1, GBD_FAULT_IO_NEVER_READY = 2, GBD_FAULT_CORRUPT_HOST_COPY = 4 };

typedef struct {
    int n, tsz;         /* quantum numbers of the sector                        */
    int rows, cols;     /* enlarged-left dim x enlarged-right dim               */
    long long offset;   /* element offset in the sector-major vector            */
} gbd_sector_info;

typedef struct {
    long long dim;          /* length of the wavefunction vector                */
    int n_sectors;
    int n_terms;            /* operator pairs (MPO states at the centre cut)    */
    int n_classes;          /* groups of terms sharing one block structure       */
    long long n_gemm;       /* sector GEMMs in one product (both phases)         */
    double useful_flops;    /* 2*m*k*n summed over those GEMMs, counted once     */
    double operator_bytes;  /* FP64 bytes of the two enlarged operator sets      */
    double mixed_bytes;     /* algorithmic HBM bytes of one GBD_MIXED_BF16X3
                               product: every operator element read once as
                               BF16 hi + lo (4 B), psi read and H psi written
                               (FP64, 8 B each)                                */
    double mixed_x_bytes;   /* overhead traffic of the two-phase form on top of
                               mixed_bytes: the phase-1 intermediate X written
                               and read once as BF16 hi + lo (8 B per element) */
    /* Device memory model of the position (bytes), from the tables: */
    double mem_operators;   /* FP64 arenas of the two enlarged operator sets    */
    double mem_planes_bf16x3; /* BF16 hi/lo operator planes (rows padded to 8)  */
    double mem_planes_sliced; /* four BF16 slice planes of the operators        */
    double mem_x_fp64;      /* phase-1 intermediate of the FP64 form            */
    double mem_x_tensor;    /* phase-1 intermediate of the tensor-core forms
                               (one buffer shared by both: four slice planes)  */
} gbd_heff_info;

typedef struct {
    double energy;
    double resid;
    int matvecs;
    int iterations;
    double ms_matvec;       /* device time spent in H_eff products               */
    int anchors;            /* mixed form: accurate anchor products taken        */
    double anchor_resid[GBD_MAX_ANCHORS]; /* exact residual norm after each anchor */
} gbd_dav_stats;

typedef struct {
    double energy_last;     /* Davidson energy at the last step of the sweep     */
    double energy_min;      /* minimum over the sweep                            */
    double max_trunc;       /* largest truncation weight in the sweep            */
    int matvecs;
    double ms_total;        /* wall time of the sweep                            */
    double ms_matvec;       /* H_eff products                                    */
    double ms_davidson;     /* Davidson excluding products                       */
    double ms_truncate;     /* density matrix, eigensolver, selection            */
    double ms_renorm;       /* enlargement + renormalisation                     */
    double ms_io_exposed;   /* host waits on IO events                           */
    double bytes_packed;    /* serialised environment bytes                      */
    double ms_pack;         /* device time of pack kernels                       */
    double useful_flops;    /* H_eff useful flops over the sweep                 */
} gbd_sweep_stats;

typedef struct {
    double energy;          /* Davidson energy (+ e_core)                        */
    double trunc_weight;    /* discarded weight of the truncation                */
    double resid;           /* final Davidson residual norm                      */
    int matvecs;
    double ms_total;        /* wall time of the step                             */
    double ms_matvec;       /* device time of the H_eff products                 */
    double ms_davidson;     /* Davidson excluding products                       */
    double ms_truncate;     /* density matrices, eigensolves, renormalisation,
                               next start vector                                */
    double ms_renorm;       /* environment loads + enlargement (pre-processing)  */
    double ms_io_exposed;   /* host waits on IO events                           */
    double useful_flops;    /* H_eff useful flops of the step                    */
    double bytes_packed;    /* environment bytes serialised to host this step    */
    double ms_device;       /* CUDA-event span of the step on the compute stream */
    int dav_status;         /* GBD_OK: Davidson converged; GBD_WARN_NOT_CONVERGED:
                               it stopped at its product limit;
                               GBD_WARN_PRECISION_FLOOR: the mixed form's
                               anchors stopped above dav_tol                */
    int anchors;            /* mixed form: anchor products of the Davidson      */
    double anchor_resid[GBD_MAX_ANCHORS]; /* exact residual norm after each anchor */
} gbd_step_stats;

/* ---------------------------------------------------------------- lifecycle */
int gbd_config_default(gbd_config* cfg);
int gbd_create(const gbd_config* cfg, gbd_ctx** out);
void gbd_destroy(gbd_ctx* ctx);
const char* gbd_last_error(void);
int gbd_version(void);

/* -------------------------------------------------------------------- model */
/* Eq. 1 with chemist integrals: H = sum h_ij a+_is a_js
 *   + 1/2 sum (ij|kl) a+_is a+_kt a_lt a_js + e_core.
 * h: L*L row-major, symmetric; eri: L^4 row-major (ij|kl), 8-fold symmetric.
 * Symmetry is checked to 1e-12 (relative to the largest element) -> GBD_ERR_ARG.
 * Builds the left/right operator sets of every cut (host tables). */
int gbd_load_integrals(gbd_ctx* ctx, int L, const double* h, const double* eri, double e_core);

/* Number of operator pairs (MPO states) at cut c (0..L). */
int gbd_mpo_bond_dim(gbd_ctx* ctx, int cut, int* dim);

/* Host-only check for tiny L (<= 5): the operator sets contracted into the
 * dense 4^L x 4^L matrix of Eq. 1 (row-major, orbital 0 most significant).
 * out must hold 4^(2L) doubles.  No device work. */
int gbd_mpo_dense(gbd_ctx* ctx, double* out, size_t cap);

/* ---------------------------------------------------------------- MPS input */
/* One site tensor (Eq. 2) as blocks.  meta: nblocks x 5 ints
 * (q_left.n, q_left.tsz, s, rows, cols); data: the blocks row-major, one after
 * another (host memory).  kind 0 = left-isometric, 1 = right-isometric.
 * Bond dimensions are inferred from the blocks and must be consistent with
 * neighbouring sites. */
int gbd_import_site(gbd_ctx* ctx, int site, int kind, int nblocks, const int* meta, const double* data);

/* The inverse of gbd_import_site (MPS checkpoints, Eq. 2): site tensor
 * `site` in the same block format.  Before the sites reach the device these
 * are the imported blocks; afterwards the current isometry, which truncations
 * (Sec. II.B step 3) replace, read back from the device, one block per
 * (q_left, s) segment.
 * With meta and data NULL only *kind, *nblocks and *data_len are written;
 * otherwise meta must hold meta_cap >= *nblocks blocks x 5 ints and data
 * data_cap >= *data_len doubles, else GBD_ERR_ARG. */
int gbd_export_site(gbd_ctx* ctx, int site, int* kind, int* nblocks, int* meta, int meta_cap, double* data,
                    size_t data_cap, size_t* data_len);

/* Builds left environments for cuts 0..b and right environments for cuts
 * L..b+2 from the imported sites (renormalisation, Sec. II.B step 3). */
int gbd_build_envs(gbd_ctx* ctx, int b);

/* ---------------------------------- sector tables (Sec. II.B, Fig. 4a) */
/* Sector table of the wavefunction at two-site position b (needs
 * gbd_build_envs or a sweep position at b).  Writes up to cap sectors to
 * out, the count to *n, and the product statistics to *info. */
int gbd_build_tables(gbd_ctx* ctx, int b, gbd_sector_info* out, int cap, int* n, gbd_heff_info* info);

/* ------------------------------- H_eff psi (Sec. II.B step 2, Eq. 3) */
/* psi_out = H_eff psi_in at position b (Sec. II.B step 2).  Vectors in the
 * sector-major layout above, FP64.  on_device = 1: both pointers are device
 * pointers; 0: host pointers (copied in and out).  precision selects the
 * product form (GBD_FP64, GBD_MIXED_BF16X3, GBD_SLICED_BF16,
 * GBD_FP64_PER_BLOCK, GBD_BF16X3_TWO_PHASE or GBD_BF16X3_FUSED).  psi_out may not alias psi_in. */
int gbd_apply_heff(gbd_ctx* ctx, int b, const double* psi_in, double* psi_out, int on_device, int precision);

/* Diagonal of H_eff at b (for preconditioning / checks), same layout. */
int gbd_heff_diagonal(gbd_ctx* ctx, int b, double* diag, int on_device);

/* ------------------------------- Davidson (Sec. II.A, Sec. II.B step 2) */
/* Lowest eigenpair of H_eff at b.  psi (host, sector-major) is the start
 * vector on entry (NULL = library's current two-site vector or random) and
 * the normalised eigenvector on exit (may be NULL).  Returns
 * GBD_WARN_NOT_CONVERGED if the product limit was reached, and in the mixed
 * form GBD_WARN_PRECISION_FLOOR if three anchors left the residual above
 * dav_tol. */
int gbd_davidson(gbd_ctx* ctx, int b, double* psi, double* energy, gbd_dav_stats* stats);

/* ------------------------------------ truncation (Sec. II.B step 3) */
/* Truncates the current two-site vector at b to at most Dmax states on the
 * enlarged left (dir = +1) or right (dir = -1) block, renormalises the
 * operators of that block (Sec. II.B step 3), and forms the next start
 * vector ("StVec", Sec. IV). */
int gbd_truncate(gbd_ctx* ctx, int b, int dir, int Dmax, double* trunc_weight);

/* ------------------------------------------------------------------ sweep */
/* nsweeps full sweeps (left-to-right over b = 0..L-3, right-to-left over
 * b = L-2..1).  Starts from the imported MPS (all sites right-isometric) or
 * from a seeded random one.  stats may be NULL; per-sweep stats are written
 * to stats[i] for i < nsweeps. */
int gbd_sweep(gbd_ctx* ctx, int nsweeps, int D, gbd_sweep_stats* stats);

/* One full two-site iteration at position b (Sec. II.B): environments made
 * resident (unpacked from host if offloaded), enlargement, Davidson from the
 * current two-site vector (random if none), truncation to D towards dir
 * (+1 right, -1 left), renormalisation, next start vector; with offload on,
 * the next needed environment is loaded and the new one saved to pinned host
 * memory asynchronously (Sec. III.B.4).  The position moves to b + dir.
 * Returns the Davidson's warning (the step still completes):
 * GBD_WARN_NOT_CONVERGED at its product limit, GBD_WARN_PRECISION_FLOOR at
 * the mixed form's anchor limit; stats->dav_status says the same. */
int gbd_step(gbd_ctx* ctx, int b, int dir, int D, gbd_step_stats* stats);

/* Copies the current two-site vector (position *b, sector-major layout) to
 * host memory.  *n gets its length; cap too small -> GBD_ERR_ARG. */
int gbd_get_psi(gbd_ctx* ctx, double* out, size_t cap, long long* n, int* b);

/* Sets the current two-site vector at position b from psi (n doubles,
 * sector-major layout of position b; host or device memory, flagged).  The
 * environments of position b must exist.  Wrong n -> GBD_ERR_ARG. */
int gbd_set_psi(gbd_ctx* ctx, int b, const double* psi, long long n, int on_device);

/* Number of this library's own kernel launches so far (all contexts). */
int gbd_launch_count(unsigned long long* count);

/* Current energies of the last sweep steps, one per step (host array). */
int gbd_step_energies(gbd_ctx* ctx, double* out, int cap, int* n);

/* ------------------ serialisation and offload (Sec. III.A, III.B.2-4) */
/* Environment ids: side 0 = left block (cut c, orbitals 0..c-1), side 1 =
 * right block (cut c, orbitals c..L-1).
 *
 * gbd_pack_env serialises one resident environment into dst (host or device
 * memory, flagged) as self-contained packages (Sec. III.B.3), one per class
 * block: a 64-byte header (magic "GBDP", version, dtype, side, cut, package
 * count and index, class, layers, q_out, q_in, rows, cols, arena offset,
 * checksum sum_i w_i (2i + 1) mod 2^64 over the payload words) followed by
 * the FP64 payload padded to 16 bytes.  If cap
 * is too small, returns GBD_ERR_ARG and writes the exact required size to
 * *bytes (size prediction, Sec. III.B.2).  */
int gbd_pack_env(gbd_ctx* ctx, int side, int cut, void* dst, size_t cap, size_t* bytes, int dst_on_device);

/* Deserialises packages (any order) into the resident environment with the
 * same id, which must exist with the same block structure (its data are
 * overwritten).  Bad magic, ids, dims or checksum -> GBD_ERR_CORRUPT. */
int gbd_unpack_env(gbd_ctx* ctx, int side, int cut, const void* src, size_t bytes, int src_on_device);

/* Imports a raw environment for pack tests: classes of layers sharing one
 * block structure.  class_meta: ncls x 3 ints (dq.n, dq.tsz, n_layers);
 * block_meta: nblk x 7 ints (class, q_out.n, q_out.tsz, q_in.n, q_in.tsz,
 * rows, cols) in canonical order (class-major); data: the blocks one after
 * another, each n_layers*rows*cols doubles (host). */
int gbd_env_import(gbd_ctx* ctx, int side, int cut, int ncls, const int* class_meta, int nblk,
                   const int* block_meta, const double* data);

/* Copies an environment's arena to host (canonical order, each block padded
 * to an even number of doubles).  *elems gets the arena size.  An
 * environment that lives only in the pinned host store (offload on) is
 * first loaded back to the device through the offload path (unpack from
 * pinned memory, package checksums verified: GBD_ERR_CORRUPT on mismatch). */
int gbd_env_export(gbd_ctx* ctx, int side, int cut, double* out, size_t cap, size_t* elems);

/* Allocation-free pack.  The paper has no counterpart to this entry point.
 *
 * Serialises a block-sparse environment that lives in caller-owned device
 * memory into caller-owned device memory, in the package format of
 * gbd_pack_env, without allocating anything: no cudaMalloc, cudaFree or
 * allocating library routine is called.  It is meant for callers that cannot
 * allocate device memory: a host runtime whose device memory is entirely
 * owned by another allocator (e.g. a framework's caching allocator that has
 * reserved the whole GPU), or a latency-critical offload thread that must
 * not take the implicit device synchronisation cudaMalloc/cudaFree can cause.
 *
 * arena: device pointer to the environment in the canonical layout of
 * gbd_env_export (blocks class-major, each padded to an even number of
 * doubles), at least the padded total of the block sizes long (the library
 * cannot check that length: a shorter arena is read out of bounds);
 * class_meta / block_meta as for gbd_env_import (host memory); side and
 * length are written into every header; dst: device memory of at least the
 * size written to *bytes (too small -> GBD_ERR_ARG with the required size).
 * arena and dst must both be 16-byte aligned device (or managed) memory,
 * else GBD_ERR_ARG before anything is launched.  stream: a cudaStream_t
 * (NULL = legacy default stream); the call returns once the stream has
 * finished the pack.
 *
 * Scratch: one file-scope device array of 8 MiB, which every GPU that loads
 * this library holds until the process exits.  Limits: 32768 packages and
 * 65536 chunks of 64 KB; larger environments -> GBD_ERR_ARG.  The first call
 * on each device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * All calls share the array, which keeps the last call's contents (the
 * checksum accumulators are cleared at the start of every call); calls that
 * overlap on the GPU (other streams, other threads) race on it. */
int gbd_pack_noalloc(int side, int length, const double* arena, int ncls, const int* class_meta, int nblk,
                     const int* block_meta, void* dst, size_t cap, size_t* bytes, void* stream);

/* Autotuner of the BF16x3 product at the current position.  The candidates
 * are phase-2 work-list shapes: split_per_sm[i] split-K work items per SM and
 * order[i] (0: items listed K range by K range across the tiles of a sector,
 * 1: tile by tile).  While active, successive BF16x3 products use candidates
 * 0, 1, ... and ms[i] records each one's device time; then the fastest is
 * chosen and cached under key, a coarse hash of the sector-size histogram
 * hist (sectors per max(rows, cols) / 64 bin, last bin open: its top bin and
 * its second moment to within 25%) and of the operator count (to within
 * 512), so the positions of one sweep region share a choice; a later
 * position with the same key takes the cached choice
 * (from_cache = 1) without trials.  default_index is the fixed shape used with
 * autotune = 0.  Fills *out for the current position while it has tuner
 * state, else with the last finished choice (position says which). */
typedef struct {
    int position, active, n_candidates, chosen, current, from_cache, default_index;
    int split_per_sm[8], order[8];
    double ms[8];
    int hist[16];
    unsigned long long key;
} gbd_tune_info;
int gbd_tune_info_get(gbd_ctx* ctx, gbd_tune_info* out);

/* Forgets every cached autotuner choice (the cache is shared by all contexts
 * of the process); the next position of each key tries the candidates again. */
int gbd_tune_reset(void);

/* Accumulated phase timers of the context in ms, in this order: enlargement
 * planning (host), enlargement kernels, renormalisation planning (host),
 * renormalisation kernels, per-sector eigensolves, Davidson anchor products
 * (host wall time, operand preparation included), tensor-core operand
 * preparation, Davidson host time (reserved), then
 * the FP64 GFLOP executed by enlargement and by renormalisation GEMMs, then
 * the tensor-core GFLOP one BF16x3 product of the last prepared H_eff issues
 * in phase 1 and in phase 2 (whole tiles, the three split products; not
 * accumulated), then the device time (ms) of all H_eff products in the
 * forms GBD_FP64, GBD_MIXED_BF16X3, GBD_SLICED_BF16, then the number of
 * products in each form, then the tensor-core GFLOP one GBD_SLICED_BF16
 * product issues (ten slice products; not accumulated), then the host wall
 * time (ms) of the tensor-core operand preparation in three parts: operator
 * splitting, planning (work lists, tensor maps), upload, then the useful
 * GFLOP of the H_eff products in each of the three forms, then the
 * renormalisation and enlargement GFLOP run on the tensor cores in the
 * sliced form (the FP64 GFLOP counters above count FP64 GEMMs only), then
 * the device time (ms, compute stream, host gaps included) of the phases of
 * gbd_step: environments resident, enlargement, Davidson, density matrices
 * and eigensolves, renormalisation, next start vector, IO scheduling, then
 * the enlargement planning (host) in three parts: coefficient links, output
 * blocks, copy and GEMM items, then the algorithmic GB the GBD_MIXED_BF16X3
 * products moved (gbd_heff_info.mixed_bytes per product: operators once,
 * psi in, H psi out), then their X overhead GB (mixed_x_bytes per product),
 * then the device time (ms) and number of GBD_FP64_PER_BLOCK products,
 * then the host wall time (ms) of environment recomputation
 * (env_recompute) and the number of environments it rebuilt, then the GB
 * written to and read back from the spill file and the host time (ms) spent
 * waiting for spill jobs (host_store_bytes), then the device time (ms) and
 * number of GBD_BF16X3_TWO_PHASE products, then of GBD_BF16X3_FUSED products.
 * *n gets the count; out may be NULL. */
int gbd_timers(gbd_ctx* ctx, double* out, int cap, int* n);

/* Offload statistics of the context so far: bytes saved to / loaded from
 * pinned host memory, host time blocked on IO events, device time of
 * gbd_pack_env calls, device time of the asynchronous save kernels (waits
 * for pending saves to finish).  Any pointer may be NULL. */
int gbd_io_stats(gbd_ctx* ctx, double* bytes_d2h, double* bytes_h2d, double* ms_exposed, double* ms_pack,
                 double* ms_save);

#ifdef __cplusplus
}
#endif
#endif /* GBDMRG_H */
