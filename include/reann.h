/*
 * reann.h -- C ABI of the GB300 (sm_103a) REANN energy/force library.
 *
 * What is computed (arXiv 2505.06711, "Efficient Parallelization of Message
 * Passing Neural Networks"):
 *   * Sec. 2.1, Eq. 1: per message-passing layer t, the embedded-atom density
 *     of every atom i, rho^t_{i,l,k} = sum_{lx+ly+lz=l} l!/(lx! ly! lz!)
 *     [ sum_{j != i, d_ij < r_c} sum_m c^t_{j,m} phi_m(d_ij) x^lx y^ly z^lz W^t_{l,m,k} ]^2
 *     with phi_m(d) = exp(-alpha (d - mu_m)^2) f_c(d), mu_m = m r_c/(N_phi - 1),
 *     f_c(d) = (cos(pi d / r_c)/2 + 1/2)^2 and (x, y, z) = r_j - r_i in A;
 *   * Sec. 2.1, Eq. 2: c^{t+1}_i = M^t_{Z_i}(rho^t_i) for t < T-1 (per-element
 *     networks F -> 64 -> 64 -> N_phi, SiLU), and after T layers the atomic
 *     energies eps_i = M^{T-1}_{Z_i}(rho^{T-1}_i), E = sum_i eps_i;
 *   * Sec. 2.2, Eqs. 3-5: forces F = -dE/dr by one reverse pass through all
 *     layers (vector-Jacobian products, never a full Jacobian);
 *   * Sec. 2.2: ONE neighbour list of radius r_c (+ skin) serves every layer,
 *     so the cost is linear in T, and ghost (periodic-image) atoms receive
 *     their owners' coefficients by an index gather once per layer instead of
 *     being recomputed (the paper's per-layer ghost-atom message refresh, Fig. 4a).
 *
 * Model shape fixed by this build: N_phi = 8 Gaussians, L = 2 (10 Cartesian
 * terms), N_orb = 16 orbitals (F = 48 features), hidden widths 64 and 64,
 * up to 8 elements, alpha r_c^2 <= 80.  Other shapes are rejected with REANN_E_ARG.
 *
 * Units: A, eV, amu, fs.  Cells are 3x3 row-major, rows = lattice vectors.
 *
 * Conventions for every entry point:
 *   * Pointers marked "dev" are CUDA device pointers (e.g. torch tensors'
 *     data_ptr()); "host" pointers are ordinary host memory.  The caller owns
 *     every pointer it passes; the library never frees caller memory and keeps
 *     no pointer to it after the call returns (it copies what it keeps).
 *   * Handles (reann_model, reann_ctx, reann_nlist) are owned by the library
 *     and released with the matching *_free.
 *   * Work is enqueued on the context's CUDA stream and is asynchronous unless
 *     stated otherwise; results in "dev" outputs are valid once that stream
 *     has reached the call's end.
 *   * Return value 0 (REANN_OK) or a negative REANN_E_* code; the message of
 *     the last failure on a context is returned by reann_last_error().
 *   * Atom order in and out is the caller's; any internal reordering is
 *     invisible.
 */
#ifndef REANN_H
#define REANN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define REANN_OK 0
#define REANN_E_ARG (-1)      /* invalid argument or unsupported model shape  */
#define REANN_E_MISMATCH (-2) /* r_c or T differs from the model's            */
#define REANN_E_NOMEM (-3)    /* device or host allocation failed             */
#define REANN_E_GEOM (-4)     /* non-finite position, coincident atoms, singular cell */
#define REANN_E_CUDA (-5)     /* a CUDA runtime call failed                   */
#define REANN_E_TIMEOUT (-6)  /* a bounded device wait ran out                */
#define REANN_E_CAPACITY (-7) /* a neighbour/ghost capacity was exceeded (rebuild) */

/* Network precisions.  The tensor-core modes round, in every 128-atom tile of
 * one element, only the deviations of a product's inputs from the tile's
 * column means; the means' products, the output layer (64 -> 8 or 1) and the
 * first reverse product are FP32, so the low precision never shifts every
 * atom alike.  All modes accumulate in FP32.                                    */
#define REANN_MLP_FP32 0   /* atomic networks in FP32 SIMT arithmetic                        */
#define REANN_MLP_BF16 1   /* tcgen05 tensor cores, BF16 operands                           */
#define REANN_MLP_BF16X3 2 /* tcgen05, every operand a BF16 hi + lo pair, 3 MMAs per K step
                              (about 16 significant bits per operand)                       */
#define REANN_MLP_FP8 3    /* tcgen05, FP8 E4M3 operands; activation rows scaled by powers
                              of two, weights per output unit by max |w| / 448              */

typedef struct reann_model reann_model;
typedef struct reann_ctx reann_ctx;
typedef struct reann_nlist reann_nlist;

/* ---------------------------------------------------------------- model --- */

/*
 * Create a model from hyper-parameters and a flat FP32 parameter vector
 * (host).  Layout (row-major, "x @ W" convention, F = (l_max+1) n_orb,
 * features ordered f = l n_orb + k):
 *   c0 [n_elem][n_phi]                      initial coefficients c^0 (Sec. 2.1)
 *   W  [T][l_max+1][n_phi][n_orb]           per-layer orbital contraction (Eq. 1)
 *   for t in 0..T-1, for e in 0..n_elem-1:  atomic network M^t_e (Eq. 2)
 *     W1 [F][h1], b1 [h1], W2 [h1][h2], b2 [h2], W3 [h2][o_t], b3 [o_t]
 *     with o_t = n_phi for t < T-1 and o_t = 1 (energy) for t = T-1.
 * n_params must equal the length implied by the shape.  Host only (no CUDA
 * call); the parameters are copied.  Errors: REANN_E_ARG.
 */
int reann_model_create(int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c, double alpha,
                       const float* params, int64_t n_params, reann_model** out);

/*
 * As reann_model_create, with the choice of features:
 *   feature_pairs = 0  Eq. 1: rho_{l,k} = sum_{a in l} w_a g_{a,k}^2, n_orb = 16, F = 48
 *   feature_pairs = 1  orbital-pair products rho_{l,(k,k')} = sum_{a in l} w_a g_{a,k} g_{a,k'}
 *                      for k <= k', n_orb = 8, F = (l_max+1) n_orb (n_orb+1)/2 = 108 (the
 *                      feature count Sec. 2.1 states), features ordered f = l 36 + p with p
 *                      enumerating (k, k') row-major; FP32 networks only
 * and the same parameter layout with these F and n_orb.  Errors: REANN_E_ARG.
 */
int reann_model_create_ex(int n_elem, int T, int n_phi, int l_max, int n_orb, int h1, int h2, double r_c,
                          double alpha, int feature_pairs, const float* params, int64_t n_params, reann_model** out);
void reann_model_free(reann_model* model);

/*
 * Load a model from a file (host only, no CUDA call): the shape of Eqs. 1-2
 * (n_elem, T, N_phi, L, N_orb, hidden widths, r_c, alpha, feature kind) and
 * the flat FP32 parameter vector laid out as for reann_model_create.
 * File layout, little-endian whatever the host:
 *   bytes  0..7   magic "REANNMDL"          bytes  8..11  uint32 version (1)
 *   bytes 12..43  int32 n_elem, T, n_phi, l_max, n_orb, h1, h2, feature_pairs
 *   bytes 44..47  uint32 reserved (0)       bytes 48..55  float64 r_c
 *   bytes 56..63  float64 alpha             bytes 64..71  int64 n_params
 *   bytes 72..    n_params float32 parameters
 *   path  host, NUL-terminated file name
 *   out   receives the new model (NULL on failure); free with reann_model_free
 * Errors: REANN_E_ARG (unreadable file, wrong magic or version, size other
 * than 72 + 4 n_params bytes, or a shape / parameter set that
 * reann_model_create_ex rejects), REANN_E_NOMEM.
 */
int reann_model_load(const char* path, reann_model** out);

/*
 * Write `model` to `path` in the layout of reann_model_load (host only; the
 * file is replaced).  Loading it gives a model with bit-identical parameters.
 * Errors: REANN_E_ARG (null argument, file not writable or write failed).
 */
int reann_model_save(const reann_model* model, const char* path);

/* -------------------------------------------------------------- context --- */

/*
 * Create an execution context on the current CUDA device: uploads the model
 * (FP32 and BF16 copies) and binds `cuda_stream` (a cudaStream_t; NULL = the
 * legacy default stream).  The model may be freed after this call.
 * Errors: REANN_E_ARG, REANN_E_NOMEM, REANN_E_CUDA.
 */
int reann_ctx_create(const reann_model* model, void* cuda_stream, reann_ctx** out);
void reann_ctx_free(reann_ctx* ctx);

/*
 * Precision of the atomic networks: REANN_MLP_FP32 (default), REANN_MLP_BF16,
 * REANN_MLP_BF16X3 or REANN_MLP_FP8 (the tensor-core modes for the 48-feature
 * models only).  The density and reverse-pass edge arithmetic stays FP32 and
 * the energy sum FP64 in every mode.  The tensor-core modes round deviations
 * from per-tile means, so their results depend (at rounding level) on which
 * atoms share a 128-atom tile: a structure evaluated alone or in a serving
 * pool gives the same bits, a decomposed list (other tiles) does not.
 * Errors: REANN_E_ARG.
 */
int reann_ctx_set_mlp_precision(reann_ctx* ctx, int precision);

/* Message of the last failure on `ctx` (static storage of the context). */
const char* reann_last_error(const reann_ctx* ctx);

/*
 * Wait for the context's stream and report device-side error flags raised
 * since the last check (coincident atoms in an evaluation -> REANN_E_GEOM,
 * neighbour/ghost capacity exceeded during a device-side rebuild ->
 * REANN_E_CAPACITY).  Synchronous.
 */
int reann_ctx_check(reann_ctx* ctx);

/*
 * Failure-detection diagnostic (no counterpart in the paper).  Every
 * mbarrier wait of the tensor-core network kernels is bounded; when one runs
 * out, the CTA records a timeout flag, waits (bounded) until the MMAs it
 * issued and its weight copy have completed, frees its tensor memory and
 * returns, and reann_ctx_check() reports REANN_E_TIMEOUT.  This call enqueues
 * on the context stream one CTA of that kind which allocates tensor memory and
 * waits `polls` times on an mbarrier that nothing ever arrives on, so the wait
 * runs out with no copy or MMA in flight and the same exit path runs.  The
 * context stays usable: the next reann_ctx_check() returns REANN_E_TIMEOUT
 * and clears the flag.  Asynchronous.
 *   polls  1 .. 2^26 polls of the barrier before the wait gives up
 * Errors: REANN_E_ARG, REANN_E_CUDA.
 */
int reann_ctx_wait_selftest(reann_ctx* ctx, int64_t polls);

/* ------------------------------------------------------- neighbour list --- */

/*
 * Build the periodic neighbour list of radius r_c + skin (Sec. 2.2: the single
 * r_c list re-used by every layer; the skin lets it survive atom motion of up
 * to skin/2, Sec. 1) and the ghost map (every periodic image within r_c + skin
 * of the cell becomes a ghost slot that points at its owner atom).
 *   n_atoms  number of atoms N >= 1
 *   pos      dev, N x 3 FP64 Cartesian positions (A), any image
 *   species  dev, N int32 element indices in [0, n_elem)
 *   cell     host, 9 FP64, rows = lattice vectors (A); must be non-singular
 *   r_c      must equal the model's cutoff (else REANN_E_MISMATCH)
 *   skin     >= 0 (A)
 * A pair (i, j, n) is listed iff |(x_j - x_i) + n.H| < r_c + skin in FP64
 * after wrapping positions into the cell, excluding only the zero-shift self
 * term (periodic self-images are neighbours).  The returned handle also holds
 * the structure's per-layer device buffers, so it stays resident for repeated
 * evaluations.  Synchronous (waits for the stream).
 * Errors: REANN_E_ARG (N < 1, species out of range), REANN_E_MISMATCH,
 * REANN_E_GEOM (non-finite position, coincident atoms, singular cell),
 * REANN_E_NOMEM, REANN_E_CUDA.
 */
int reann_build_nlist(reann_ctx* ctx, int64_t n_atoms, const double* pos, const int32_t* species, const double* cell,
                      double r_c, double skin, reann_nlist** out);
void reann_nlist_free(reann_nlist* nl);

/*
 * Rebuild the list of `nl` for new positions (dev, N x 3 FP64) on the device,
 * re-using the capacities sized by reann_build_nlist: no allocation and no
 * host synchronisation, so it can be enqueued between evaluations or inside
 * a captured CUDA graph.  Same pair definition as reann_build_nlist.  If atom
 * motion needs more ghost slots or row entries than were sized, the affected
 * entries are dropped and reann_ctx_check() reports REANN_E_CAPACITY; build a
 * new list then.  Asynchronous.  Errors: REANN_E_ARG, REANN_E_CUDA.
 * Repeated calls with the same arguments are replayed as one CUDA graph (the
 * first runs directly, the second is captured) on a library-owned stream
 * ordered after and before the context stream; with reann_ctx_profile on,
 * every call launches its kernels directly.  Every 8th rebuild (counted on the
 * device, MD rebuilds included) also re-sorts the atoms' internal order (by
 * element and cell bin, for locality); the others keep the order of the last
 * sort.  The list (pairs, ghosts) is the same either way.
 */
int reann_nlist_rebuild(reann_ctx* ctx, reann_nlist* nl, const double* pos);

/*
 * Sizes (host outputs, each nullable): atoms, ghost slots in use, listed
 * (i, j, n) entries within r_c + skin, and the entries within r_c found by the
 * last evaluation (0 before the first).  Synchronous.
 */
int reann_nlist_info(const reann_nlist* nl, int64_t* n_atoms, int64_t* n_ghosts, int64_t* n_pairs, int64_t* n_live);

/*
 * Copy the list to host arrays as (i, j, n) triples in the caller's atom
 * order with n relative to the caller's (unwrapped) positions at build time:
 * r_ij = x_j + n.H - x_i.  Writes min(cap, count) entries; *count = total.
 * Synchronous.  Errors: REANN_E_ARG.
 */
int reann_nlist_export(reann_ctx* ctx, const reann_nlist* nl, int64_t cap, int32_t* i, int32_t* j, int32_t* n,
                       int64_t* count);

/* ------------------------------------------------- spatial decomposition --- */

/*
 * The paper's parallel scheme (Sec. 2.2, Figs. 3-5) as virtual ranks on one
 * device.  The cell is cut into ranks[0] x ranks[1] x ranks[2] subdomains in
 * fractional coordinates (ranks host, each 1..64).  Rank r owns the atoms of
 * its subdomain (local atoms) and holds a ghost slot for every atom or
 * periodic image within r_c + skin of one of its local atoms that is not a
 * zero-shift local atom of r (owned by another rank, or an image); its
 * neighbour rows reference only its own local atoms and ghost slots.  The
 * returned list evaluates through reann_energy_forces unchanged: before each
 * layer every ghost slot receives its owner's coefficients (the per-layer
 * exchange of Fig. 4a), and in the reverse pass its owner's bbar (the ghost
 * gradient exchange of Sec. 2.2 in vector-Jacobian-product form), so the halo
 * is r_c + skin for every T.  Rows keep the single-domain entry order and ghost
 * slots hold bit-identical copies, so forces equal the single-domain list's
 * bit for bit (energies to the order of the FP64 sum).  Other arguments as
 * reann_build_nlist; synchronous (the subdomain bookkeeping runs on the host
 * once).  Such a list is not rebuilt in place: reann_nlist_rebuild, an
 * automatic rebuild in reann_energy_forces_host and reann_md_step return
 * REANN_E_ARG.  Errors: as reann_build_nlist; REANN_E_ARG for bad ranks.
 */
int reann_build_nlist_decomposed(reann_ctx* ctx, int64_t n_atoms, const double* pos, const int32_t* species,
                                 const double* cell, double r_c, double skin, const int32_t ranks[3],
                                 reann_nlist** out);

/*
 * Per-rank sizes of a decomposed list (a single-domain list reports one rank):
 * *n_ranks, and for each rank (host arrays of n_ranks entries, each nullable)
 * its local atoms, ghost slots, and ghost slots owned by another rank (the
 * slots the per-layer exchange fills across ranks).  Synchronous.
 */
int reann_decomp_info(const reann_nlist* nl, int32_t* n_ranks, int64_t* local, int64_t* ghosts, int64_t* remote);

/* ------------------------------------------------------------ evaluation --- */

/*
 * Energy and forces of the structure of `nl` at positions `pos` (Eqs. 1-5).
 *   pos          dev, N x 3 FP64 (A); atoms must have moved less than skin/2
 *                since the list was built (the caller decides when to rebuild)
 *   T            number of message-passing layers; must equal the model's
 *   energy       dev, 1 FP64: E = sum_i eps_i (eV), summed in FP64
 *   forces       dev, N x 3 FP32: F = -dE/dr (eV/A)
 *   atom_energy  dev, N FP32 per-atom energies eps_i, or NULL
 * Asynchronous.  Coincident atoms are reported by reann_ctx_check().
 * Repeated calls with the same pointers, T and network precision are replayed
 * as one CUDA graph, as for reann_nlist_rebuild.
 * Errors: REANN_E_ARG, REANN_E_MISMATCH, REANN_E_CUDA.
 */
int reann_energy_forces(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy, float* forces,
                        float* atom_energy);

/*
 * reann_energy_forces plus the virial.  Eq. 1 is the only place positions
 * enter, through the edge vectors r_e (periodic images included), so
 *   virial  dev, 3 x 3 FP64 row-major: W_ab = -sum_e (dE/dr_e)_a (r_e)_b
 *           = -dE/d eps_ab for a homogeneous strain x -> (I + eps) x of the
 *           positions and the cell (the configurational part of the stress
 *           times the volume: sigma = -(W + kinetic) / V); summed in FP64
 *   atom_virial  dev, N x 9 FP32 per-atom share (each directed edge e = (i, j)
 *           of every layer assigned to its centre i), caller order, or NULL
 * The first call allocates the per-atom buffer (N x 36 B), later calls do not.
 * Asynchronous.  Errors: as reann_energy_forces; REANN_E_NOMEM.
 */
int reann_energy_forces_virial(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy,
                               float* forces, float* atom_energy, double* virial, float* atom_virial);

/*
 * Same as reann_energy_forces with HOST buffers: copies pos (host, N x 3
 * FP64) to the device, rebuilds the neighbour list on the device (always if
 * `rebuild` is non-zero, otherwise only when an atom moved more than skin/2
 * since the last build), evaluates, and copies energy (host, 1 FP64) and
 * forces (host, N x 3 FP32, caller order) back.  Synchronous; includes the
 * reann_ctx_check() of the evaluation.  Pinned host memory makes the copies
 * DMA transfers; pageable memory works but is slower.
 */
int reann_energy_forces_host(reann_ctx* ctx, reann_nlist* nl, const double* pos, int T, double* energy,
                             float* forces, int rebuild);

/* ---------------------------------------------------------------- serving --- */

/*
 * Continuous-batching pool: many independent structures resident on the
 * device and evaluated together by one launch sequence (one evaluation of the
 * paper's path, Sec. 2.1-2.2, over all of them), with per-structure offsets.
 *   reann_serve_create  reserve a pool of max_atoms owned slots, max_ghosts
 *                       ghost slots, max_structures structures and neighbour
 *                       rows of `stride` entries on ctx's device; its device
 *                       memory (about 3.5 kB per atom at T = 3 plus 8 B per row
 *                       entry) is the admission budget.  Synchronous.
 *   reann_serve_submit  build the structure's list with build_ctx (its own
 *                       stream, so builds overlap pool launches in flight),
 *                       then, if free owned and ghost ranges and a structure
 *                       slot remain, pack it into the pool (on the pool's
 *                       stream, after any launch already enqueued) and return
 *                       its slot; otherwise REANN_E_NOMEM (admission refused:
 *                       retry after a release).  pos/species dev, caller
 *                       order; cell host 9 FP64.  Rows longer than `stride`:
 *                       REANN_E_CAPACITY.
 *   reann_serve_launch  evaluate every structure submitted since the last
 *                       launch: energies[slot] (dev FP64, max_structures
 *                       entries) and forces (dev FP32, (max_atoms + 1) x 3:
 *                       rows [offset, offset + n) of each launched slot in its
 *                       caller order, the last row is scratch).  `slots`
 *                       (host, max_structures, nullable) and *count receive the
 *                       launched slots.  The launch covers only the pool's
 *                       rows and ghost slots below the launched structures'
 *                       highest ones, rounded up to a size class (the pool's
 *                       capacity divided by 1, 2, 4, ... 128, at least 2,048
 *                       rows), so its cost follows the work, not the pool's
 *                       size.  Every class is captured as a CUDA graph on the
 *                       first launch (per precision and output pointers; that
 *                       launch itself runs directly) and replayed afterwards;
 *                       submissions take the lowest free ranges, which keeps
 *                       the classes small.  Asynchronous: the
 *                       context stream waits for it.  A slot is evaluated
 *                       once; later launches leave its energy entry and force
 *                       rows untouched until it is released.
 *   reann_serve_release free a slot's ranges once its results were read
 *                       (REANN_E_ARG for a slot not in use).
 * The reann_serve_* calls on one pool are thread-safe: several threads, each
 * with its own build_ctx, may submit while another launches and releases; the
 * builds themselves run concurrently.
 * Each structure's arithmetic is independent of its batch mates (own rows,
 * own network tiles, own FP64 energy segment), so results are bitwise the same
 * alone and in any mix.
 */
typedef struct reann_serve reann_serve;
int reann_serve_create(reann_ctx* ctx, int64_t max_atoms, int64_t max_ghosts, int max_structures, int stride,
                       reann_serve** out);
void reann_serve_free(reann_serve* srv);
int reann_serve_submit(reann_serve* srv, reann_ctx* build_ctx, int64_t n_atoms, const double* pos,
                       const int32_t* species, const double* cell, double skin, int* slot);
int reann_serve_launch(reann_serve* srv, double* energies, float* forces, int* slots, int* count);
int reann_serve_release(reann_serve* srv, int slot);
/* atom offset and size of a used slot (host outputs, nullable) */
int reann_serve_slot(reann_serve* srv, int slot, int64_t* atom_offset, int64_t* n_atoms);
/* largest free owned range, largest free ghost range, free structure slots */
int reann_serve_usage(reann_serve* srv, int64_t* free_atoms, int64_t* free_ghosts, int* free_slots);

/* ------------------------------------------------------ no-allocation sum --- */

/*
 * Total energy E = sum_i eps_i in FP64 from per-atom energies the caller
 * already holds, without allocating any device memory.  The paper has no
 * counterpart.  It exists for callers that must not allocate when they need
 * the total: force back-ends hosted as plugins by a molecular-dynamics engine
 * whose force callback may not allocate (the engine owns the device-memory
 * budget and its pools), and latency-critical callbacks that avoid cudaMalloc
 * because it can synchronise the device.
 *   atom_energy  dev, n_atoms FP32 (e.g. the atom_energy output of
 *                reann_energy_forces); NULL only when n_atoms == 0
 *   n_atoms      0 <= n_atoms <= reann_energy_sum_noalloc_max_atoms()
 *                (8,388,608); larger sizes return REANN_E_CAPACITY, no work
 *   energy       dev, 1 FP64, overwritten
 *   cuda_stream  cudaStream_t to enqueue on (NULL = legacy default stream)
 * The sum is FP64 throughout (blocks of 2,048 atoms, then the block sums);
 * reann_energy_forces groups the same FP64 additions differently (per network
 * tile, in its internal atom order), so the two totals agree to FP64 rounding,
 * not bit for bit.
 * Scratch is a fixed 32 KiB array inside the library, held by every GPU that
 * loads it until the process exits.  The first call on each device looks up
 * that array's device address (cudaGetSymbolAddress) and caches it for the
 * life of the process; make that first call before any stream capture.  After
 * cudaDeviceReset on a device the cached address is stale: do not call this
 * entry point on that device again in the same process.  All calls share the
 * array and it keeps the last call's contents (each call writes every entry it
 * reads): calls that overlap on the GPU race and must be serialised by the
 * caller.  Asynchronous.
 * Errors: REANN_E_ARG, REANN_E_CAPACITY, REANN_E_CUDA (returned directly; no
 * context message).  REANN_E_CUDA reports an error that the CUDA runtime
 * returned at one of this call's launches; it can also be a pending error left
 * by earlier asynchronous work on the same device.
 */
int reann_energy_sum_noalloc(const float* atom_energy, int64_t n_atoms, double* energy, void* cuda_stream);
int64_t reann_energy_sum_noalloc_max_atoms(void);

/* ------------------------------------------------------------- profiling --- */

/*
 * Per-region event profile: when enabled, every region of the evaluation
 * (neighbour rebuild, position refresh, live-edge filter, coefficient init,
 * ghost gathers, density forward, networks forward, energy sum, networks
 * backward, bbar, density adjoint, output scatter) is bracketed by CUDA events
 * on the context's stream.  Enabling or disabling resets the totals.
 * reann_ctx_profile_read() waits for the stream and writes, per region, the
 * summed device time (ms) and the number of timed launches into arrays of
 * reann_profile_regions() entries; reann_profile_region_name() names them.
 */
int reann_ctx_profile(reann_ctx* ctx, int enable);
int reann_profile_regions(void);
const char* reann_profile_region_name(int region);
int reann_ctx_profile_read(reann_ctx* ctx, double* total_ms, int64_t* launches);

/*
 * NVE molecular dynamics: n_steps velocity-Verlet steps of dt_fs (fs) with
 * REANN forces (the benchmark systems' MD of Sec. 2.3 / 4.1 without a
 * thermostat), positions and velocities integrated in FP64:
 *   v += dt/2 F/m;  x += dt v;  if any atom moved more than skin/2 since the
 *   last build: rebuild the list on the device;  F = -dE/dx;  v += dt/2 F/m.
 *   pos    dev, N x 3 FP64 (A), caller order, updated in place
 *   vel    dev, N x 3 FP64 (A/fs), updated in place
 *   mass   dev, N FP64 (amu)
 *   e_pot  dev, n_steps FP64: E after each step (eV), or NULL
 *   e_kin  dev, n_steps FP64: kinetic energy after each step (eV), or NULL
 * The first call (and any call whose pointers, dt, n_steps or network
 * precision differ from the previous one) evaluates the starting forces and
 * captures one step as a CUDA graph on a library-owned stream, ordered after
 * the context stream; every step is then one graph launch, the rebuild being
 * a device-side decision.  Asynchronous with respect to the host; the context
 * stream waits for the steps.  Capacity overflow during a rebuild is reported
 * by reann_ctx_check() (REANN_E_CAPACITY: build a new list).
 * Errors: REANN_E_ARG, REANN_E_NOMEM, REANN_E_CUDA.
 */
int reann_md_step(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt_fs,
                  int n_steps, double* e_pot, double* e_kin);

/*
 * NVT molecular dynamics (the paper's MD ensemble, Sec. 4.1): as reann_md_step
 * with one Nose-Hoover thermostat at temperature_k (K) with time constant
 * tau_fs (fs): friction xi' = (2K - g kB T)/Q, Q = g kB T tau^2, g = 3N - 3,
 * integrated by a time-reversible splitting (a thermostat half step before
 * the first and after the second velocity half-kick).  The thermostat state
 * (xi, eta) belongs to the list and carries over between calls.
 *   e_bath  dev, n_steps FP64: Q xi^2 / 2 + g kB T eta after each step (eV),
 *           or NULL; E + K + e_bath is the conserved quantity
 * Errors: REANN_E_ARG (also for T or tau not > 0), REANN_E_NOMEM, REANN_E_CUDA.
 */
int reann_md_step_nvt(reann_ctx* ctx, reann_nlist* nl, double* pos, double* vel, const double* mass, double dt_fs,
                      int n_steps, double temperature_k, double tau_fs, double* e_pot, double* e_kin, double* e_bath);

/* Steps run by the last reann_md_step call and neighbour-list rebuilds since the
 * first one (host outputs, nullable).  Synchronous. */
int reann_md_info(reann_ctx* ctx, const reann_nlist* nl, int64_t* steps, int64_t* rebuilds);

/*
 * Per-layer intermediates of the last evaluation of `nl`, in caller order
 * (inspection and testing): rho (dev, N x F FP32, F the model's feature count)
 * and c (dev, N x N_phi FP32)
 * of layer `layer` in [0, T).  Either output may be NULL.  Asynchronous.
 */
int reann_get_layer(reann_ctx* ctx, const reann_nlist* nl, int layer, float* rho, float* coef);

#ifdef __cplusplus
}
#endif

#endif /* REANN_H */
