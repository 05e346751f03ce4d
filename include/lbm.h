/*
 * lbm.h -- C ABI of the sparse-lattice D3Q19 TRT stream-collide library.
 *
 * The library implements the propagation-plus-collision step of the lattice
 * Boltzmann method on a sparse lattice with indirect addressing, as studied in
 * Wittmann, Zeiser, Hager, Wellein, "Modeling and analyzing performance for
 * highly optimized propagation steps of the lattice Boltzmann method on sparse
 * lattices": only fluid nodes are stored, in a 1-D vector ordered by an
 * enumeration function (Sect. 1, Sect. 5.6); an adjacency list gives the 18
 * neighbours of every node (Sect. 4, "Loop Balance"); reduced indirect
 * addressing (RIA) replaces it by a run-length table where consecutive nodes
 * share a shifted access pattern (Sect. 4.1).  Three storage forms are
 * offered: the two-grid one-step form OS-NT and the single-grid AA pattern
 * (Sect. 4), and the single-grid Esoteric Twist the paper names (Sect. 1,
 * Sect. 4).  A lattice can also be cut into chunks that step separately with a
 * ghost-PDF exchange, the distributed form of Sect. 6.
 *
 * Conventions that hold for every call below:
 *  - Every function returns an int status (LBM_OK = 0 on success).  Errors
 *    are never fatal; lbm_last_error() returns a message for the calling
 *    thread's most recent failure.
 *  - Device memory is always owned by the caller and passed as a raw device
 *    pointer.  Host-side tables are owned by the opaque lbm_lattice handle.
 *  - Threads: calls on different handles are independent.  Calls that change
 *    a handle (uploads, and the first Esoteric Twist query, which derives its
 *    tables) must not run concurrently with other calls on the same handle;
 *    stepping calls only read the handle and may overlap.
 *  - Host tables are built with std::thread workers: as many as the hardware
 *    threads (at most 64), or the environment variable LBM_HOST_THREADS
 *    (1..256) when set.  The tables never depend on the thread count.
 *  - Device work is enqueued on `stream` (a cudaStream_t passed as void*;
 *    NULL selects the legacy default stream) and is asynchronous: a call
 *    returns once the kernels are queued.  Launch errors are reported as
 *    LBM_ERR_CUDA.
 *  - D3Q19 directions: 0 = rest; 1..6 = +x,-x,+y,-y,+z,-z; then the face
 *    diagonals in opposite pairs 7 (1,1,0) 8 (-1,-1,0) 9 (1,-1,0) 10 (-1,1,0)
 *    11 (1,0,1) 12 (-1,0,-1) 13 (1,0,-1) 14 (-1,0,1) 15 (0,1,1) 16 (0,-1,-1)
 *    17 (0,1,-1) 18 (0,-1,1).  The opposite of 2k-1 is 2k.
 *  - PDF arrays are structure-of-arrays: element (i, n) of a grid lives at
 *    pdf[i * Npad + n], Npad = N rounded up to a multiple of 128.  The element
 *    type is double (LBM_F64 and LBM_F64_DF), float (LBM_F32) or a 16-bit
 *    IEEE half (LBM_F16S).  With params->shifted the stored value is f_i - w_i * rho0
 *    (LBM_F16S always stores half((f_i - w_i rho0) * f16_scale)).
 *  - "Canonical" state F[i][n]: the pre-collision PDFs after the last step,
 *    FP64, unshifted, dense [19][N].
 *  - Grid layouts: LBM_LAYOUT_OSNT = an OS-NT grid (holds post-collision
 *    PDFs; the canonical state is one pull gather away); LBM_LAYOUT_AA_EVEN =
 *    the AA grid after an even number of steps (holds the canonical state);
 *    LBM_LAYOUT_AA_ODD = the AA grid after an odd number of steps;
 *    LBM_LAYOUT_ET_EVEN / LBM_LAYOUT_ET_ODD = the Esoteric Twist grid after
 *    an even / odd number of steps.  Esoteric Twist grids have the stride
 *    Spad of lbm_et_info instead of Npad: they also hold phantom locations.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LBM_API __attribute__((visibility("default")))
#else
#define LBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define LBM_OK 0
#define LBM_ERR_ARG 1          /* invalid argument, size, pointer or state        */
#define LBM_ERR_ALLOC 2        /* host allocation failed                           */
#define LBM_ERR_CUDA 3         /* a CUDA runtime call or kernel launch failed      */
#define LBM_ERR_TABLE 4        /* lattice tables violate an invariant             */
#define LBM_ERR_UNSUPPORTED 5  /* valid request the library does not implement    */
#define LBM_ERR_NONFINITE 6    /* a reduction met NaN or Inf                       */

/* ---- enumerations ----------------------------------------------------------- */
#define LBM_ENUM_LEX 0       /* lexicographic order with blocking factor B (Sect. 5.6) */
#define LBM_ENUM_HILBERT 1   /* Hilbert space-filling curve (Sect. 5.6)                */

#define LBM_F64 0            /* double storage, double collision; the step kernels
                                take the moments as exact integer sums rounded once
                                to double (lbm_exact_moments_host)                */
#define LBM_F32 1            /* float storage, float collision                       */
#define LBM_F16S 2           /* half storage of (f - w rho0) * f16_scale, float math */
#define LBM_F64_DF 3         /* double storage (same grids as LBM_F64); the step's
                                collision runs in double-float arithmetic (pairs of
                                floats, ~48 bits) on the FP32 pipe.  Only the step
                                kernels differ; every other call treats the grid as
                                LBM_F64. */

#define LBM_LAYOUT_OSNT 0
#define LBM_LAYOUT_AA_EVEN 1
#define LBM_LAYOUT_AA_ODD 2
#define LBM_LAYOUT_ET_EVEN 3 /* Esoteric Twist grid after an even number of steps */
#define LBM_LAYOUT_ET_ODD 4  /* Esoteric Twist grid after an odd number of steps  */

#define LBM_TABLES_ADJ 1     /* full adjacency list, 18 x int32 per node (Sect. 4)   */
#define LBM_TABLES_RIA 2     /* RIA run table (Sect. 4.1)                            */
#define LBM_TABLES_ET 4      /* Esoteric Twist locations and link mask, 28 B per node */

#define LBM_MARK_WALL (-1)   /* adjacency marker: halfway bounce-back               */
#define LBM_MARK_INLET (-2)  /* adjacency marker: pressure inlet face x = -1         */
#define LBM_MARK_OUTLET (-3) /* adjacency marker: pressure outlet face x = X         */

typedef struct lbm_lattice lbm_lattice;   /* opaque, owned by the library */

/* Boundary conditions of the box faces.  periodic[a] wraps axis a (x, y, z).
 * A non-periodic face is a halfway bounce-back wall, except the two x faces
 * when x_pressure is set: then x = -1 is a pressure inlet and x = X an outlet
 * (anti-bounce-back).  x may not be both periodic and a pressure axis. */
typedef struct {
  int periodic[3];
  int x_pressure;
} lbm_bc;

/* Physical and storage parameters of a step.
 *  omega_plus  TRT even relaxation rate lambda+ (0 < omega_plus < 2)
 *  magic       TRT magic parameter Lambda = (1/l+ - 1/2)(1/l- - 1/2) > 0
 *  g[3]        body-force density per unit mass (force = rho g)
 *  rho0        reference density of the shifted storage and of init
 *  rho_in, rho_out  densities imposed at the pressure inlet / outlet
 *  shifted     nonzero: store f - w_i rho0 (required for LBM_F16S)
 *  f16_scale   LBM_F16S scale (e.g. 1024); ignored otherwise */
typedef struct {
  double omega_plus;
  double magic;
  double g[3];
  double rho0;
  double rho_in;
  double rho_out;
  int shifted;
  double f16_scale;
} lbm_params;

/* Message describing the calling thread's most recent failed call ("" if none).
 * The pointer stays valid until the next failing call on the same thread. */
LBM_API const char* lbm_last_error(void);

/* ---- lattice construction (host) -------------------------------------------- */

/* Build the sparse lattice of a voxel geometry: enumerate the fluid voxels,
 * fill the adjacency list and the RIA run table.
 * Sect. 1 and Sect. 5.6 (enumeration by LS with blocking factor B or by the
 * Hilbert curve), Sect. 4 "Loop Balance" (adjacency list, Fig. 2a), Sect. 4.1
 * (RIA, Fig. 2b).
 *  solid   host array [Z][Y][X] (x fastest), nonzero = solid; not retained.
 *  X,Y,Z   box size, each >= 1, X*Y*Z < 2^40; at most 2^31-1 fluid nodes.
 *  bc      boundary conditions (see lbm_bc).
 *  enumeration  LBM_ENUM_LEX or LBM_ENUM_HILBERT.
 *  block_B LS blocking factor (>= 1; 1 = plain lexicographic); ignored for
 *          Hilbert.
 *  out     receives the new handle; free it with lbm_free_lattice.
 * Node order, adjacency entries and runs are defined exactly (bit-exact
 * tables): LS sorts by (z/B, y/B, x/B, z, y, x); Hilbert by Skilling's index
 * with bits interleaved x, y, z from the most significant level on a 2^k cube.
 * Returns LBM_ERR_ARG for bad sizes/pointers, LBM_ERR_ALLOC on host OOM. */
LBM_API int lbm_build_lattice(const uint8_t* solid, int X, int Y, int Z, const lbm_bc* bc,
                      int enumeration, int block_B, lbm_lattice** out);

/* Build a lattice from a caller-supplied adjacency list instead of voxels
 * (Sect. 4, Fig. 2a: the list is the lattice).  adj is host [18][N], entries
 * a node index in [0, N) or a marker -1/-2/-3; node_xyz (host [N][3], may be
 * NULL) is kept for export.  The RIA table is derived from adj.  Call
 * lbm_validate_tables to check the list before use. */
LBM_API int lbm_lattice_from_adjacency(int64_t N, const int32_t* adj, const int32_t* node_xyz,
                               lbm_lattice** out);

/* Build a lattice whose node order the caller gives: node_xyz (host [N][3],
 * x y z) must list every fluid voxel of `solid` exactly once.  Adjacency and
 * RIA tables follow as in lbm_build_lattice.  Used for the paper's two-stage
 * renumbering (Sect. 6.1) and any other enumeration. */
LBM_API int lbm_build_lattice_ordered(const uint8_t* solid, int X, int Y, int Z, const lbm_bc* bc,
                                      const int32_t* node_xyz, int64_t N, lbm_lattice** out);

/* The paper's two-stage renumbering (Sect. 1, Sect. 6.1): cut the current node
 * order into P equal chunks (chunk p = nodes [N p / P, N (p+1) / P)), as the
 * paper partitions the adjacency list among processes, and re-sort every chunk
 * lexicographically (x fastest, B = 1).  Writes the new order to node_xyz_out
 * (host [N][3]); build it with lbm_build_lattice_ordered. */
LBM_API int lbm_renumber_partitions(const lbm_lattice* lat, int P, int32_t* node_xyz_out);

/* Ghost PDFs of the same P-chunk partitioning: ghost_pdfs[p] (host int64 [P])
 * counts the pulls of chunk p's nodes from fluid nodes in other chunks, i.e.
 * the PDFs chunk p must receive every step (Sect. 6, communication volume). */
LBM_API int lbm_partition_ghosts(const lbm_lattice* lat, int P, int64_t* ghost_pdfs);

/* Release a handle (NULL is ignored).  Device buffers are the caller's. */
LBM_API void lbm_free_lattice(lbm_lattice* lat);

/* ---- partitions with a ghost-PDF exchange (Sect. 6, Sect. 6.1) --------------------
 * The distributed form of the step: the node vector is cut into the same P
 * chunks as above and each chunk is updated on its own grids, after receiving
 * the PDFs its nodes pull from other chunks.  One GPU holds all P grids here
 * (the exchange kernel copies between them); the tables and the exchange are
 * those a one-chunk-per-GPU run would use.
 *
 * Chunk p becomes an ordinary lattice handle ("local lattice") with N_p =
 * |chunk| nodes in the chunk's order, followed by ghost slots: a pull of PDF i
 * from a node of another chunk points at slot N_p + k, k counting that
 * chunk's earlier such pulls of direction i in node order.  The local
 * lattice's Npad covers the slots, and its RIA table is derived from the local
 * adjacency list, so lbm_step_osnt, lbm_step_aa (one AA step at a time
 * between exchanges), lbm_init_equilibrium and lbm_load_canonical (layout
 * LBM_LAYOUT_AA_EVEN) work on it unchanged.  lbm_canonical_pdfs and
 * lbm_macroscopic in the OS-NT or AA-odd layout gather through the ghost
 * slots, so they need the ghosts filled first.  The objective, adjoint and
 * checkpointed-gradient calls, and lbm_load_canonical in a pulled layout,
 * return LBM_ERR_UNSUPPORTED on a local lattice. */
typedef struct lbm_partitioning lbm_partitioning;

#define LBM_HALO_OSNT 0        /* before an OS-NT step: fill slot s of array i from the owner's P_i  */
#define LBM_HALO_AA_GATHER 1   /* before an AA odd step: fill slot s of array inv(i)                  */
#define LBM_HALO_AA_SCATTER 2  /* after an AA odd step: return slot s of array inv(i) to the owner     */

/* Partition `lat` into P chunks [N p / P, N (p+1) / P), 1 <= P <= max(N, 1),
 * and build the local lattices and the exchange table on the host.  The
 * result does not refer to `lat` afterwards.  LBM_ERR_UNSUPPORTED if a chunk
 * needs more than 2^27 nodes plus ghost slots or the lattice more than 2^31
 * ghost PDFs. */
LBM_API int lbm_partition_build(const lbm_lattice* lat, int P, lbm_partitioning** out);

/* Release a partitioning and its local lattices (NULL is ignored). */
LBM_API void lbm_free_partitioning(lbm_partitioning* part);

/* Chunk p: its first node in the partitioned lattice, its node count, its
 * ghost PDFs per exchange (equal to lbm_partition_ghosts) and its ghost slots
 * per direction array (the largest per-direction count).  Outputs may be NULL. */
LBM_API int lbm_partition_info(const lbm_partitioning* part, int p, int64_t* first_node, int64_t* N_p,
                               int64_t* ghost_pdfs, int64_t* ghost_slots);

/* The local lattice of chunk p, owned by `part` (never free it; it lives as
 * long as `part`).  Upload its tables with lbm_lattice_upload as usual. */
LBM_API int lbm_partition_local(lbm_partitioning* part, int p, lbm_lattice** local);

/* Chunk p's ghost PDFs (host int32 arrays of ghost_pdfs entries, any may be
 * NULL), in exchange order: owner chunk, pulled direction i (1..18), local
 * slot, and the source node as a local index of the owner. */
LBM_API int lbm_partition_export_ghosts(const lbm_partitioning* part, int p, int32_t* src_part, int32_t* dir,
                                        int32_t* slot, int32_t* src_node);

/* Check that every local adjacency list, read through the ghost map, equals
 * `lat`'s rows of its chunk, that the ghost map is in range and one-to-one,
 * and that each local RIA table decodes to its adjacency list.  LBM_ERR_TABLE
 * names the first violation. */
LBM_API int lbm_partition_validate(const lbm_partitioning* part, const lbm_lattice* lat);

/* Bytes of the caller-owned device buffer for the exchange table (8 B per
 * ghost PDF plus per-CTA and per-chunk words). */
LBM_API int lbm_halo_table_bytes(const lbm_partitioning* part, size_t* bytes);

/* Copy the exchange table into dev (device, 256-byte aligned, >=
 * lbm_halo_table_bytes) on `stream`; same ownership rules as
 * lbm_lattice_upload. */
LBM_API int lbm_halo_upload(lbm_partitioning* part, void* dev, size_t bytes, void* stream);

/* One exchange of all chunks' ghost PDFs on `stream` (one launch).  grids:
 * DEVICE array of P pointers, grids[p] = chunk p's grid ([19][Npad_p] of the
 * precision's element type).  mode: LBM_HALO_*.  A sequence for OS-NT is
 * exchange(OSNT, src grids), then the P steps src -> dst; for the AA pattern,
 * the P even steps, exchange(AA_GATHER), the P odd steps,
 * exchange(AA_SCATTER).  Asynchronous; LBM_ERR_ARG if the table was not
 * uploaded. */
LBM_API int lbm_halo_exchange(const lbm_partitioning* part, int prec, void* const* grids, int mode, void* stream);

/* `steps` AA steps of all chunks from parity start_parity: even steps are the
 * P local even steps; odd steps are exchange(AA_GATHER), the P odd steps and
 * exchange(AA_SCATTER).  grids_host: host array of the P chunk grids; grids_dev:
 * device array holding the same P pointers.  s: Brinkman field of the whole
 * partitioned lattice (device float [N], chunk p uses s + first_node(p)) or
 * NULL.  ria selects the addressing as for lbm_step_aa.  Asynchronous with
 * respect to `stream`: the chunks of one step run concurrently on up to 16
 * side streams that the partitioning creates on its first run (on the device
 * current then, which all later runs must use) and joins back into `stream`
 * before the next exchange, so work queued on `stream` before and after the
 * call is ordered with it as usual.  The side streams belong to the
 * partitioning: runs of one partitioning must not overlap in time (issue them
 * on one stream, or wait for the previous run); separate partitionings are
 * independent. */
LBM_API int lbm_partition_run_aa(const lbm_partitioning* part, int prec, const lbm_params* params,
                                 void* const* grids_host, void* const* grids_dev, const float* s, int start_parity,
                                 int steps, int ria, void* stream);

/* `steps` OS-NT steps of all chunks, ping-ponging two grid sets: grids_host /
 * grids_dev hold 2P pointers, set 0 (entries 0..P-1) the current source.  Step
 * k is exchange(OSNT) on set k mod 2, then the P steps from set k mod 2 into
 * the other set; after an odd count set 1 holds the state.  Streams as for
 * lbm_partition_run_aa. */
LBM_API int lbm_partition_run_osnt(const lbm_partitioning* part, int prec, const lbm_params* params,
                                   void* const* grids_host, void* const* grids_dev, const float* s, int steps,
                                   int ria, void* stream);

/* Sizes of a lattice.  Any output pointer may be NULL.  run_hist[b], b = 0..32,
 * counts RIA runs of length in [2^b, 2^(b+1)). */
LBM_API int lbm_lattice_info(const lbm_lattice* lat, int64_t* N, int64_t* Npad, int64_t* R,
                     int64_t* run_hist);

/* Copy the host tables out (bit-exact comparison).  Any pointer may be NULL.
 *  node_xyz [N][3] (x, y, z) of each node in enumeration order
 *  adj      [18][N] pull source of f_{i}, i = 1..18, node index or marker
 *  run_start [R+1]  first node of each run, run_start[R] = N
 *  run_adj  [18][R] adjacency entries of each run's first node */
LBM_API int lbm_export_tables(const lbm_lattice* lat, int32_t* node_xyz, int32_t* adj,
                      int32_t* run_start, int32_t* run_adj);

/* The run slot tables that the RIA steps read (Sect. 4.1's run table with each
 * entry resolved to a flat index of the [19][Npad] grid), for bit-exact
 * comparison on the host.  With r a run, h its first node and a = run_adj[i][r]:
 *  kind 0 (AA odd step):  slot(i, r) = inv(i) Npad + a  (a >= 0),  i Npad + h (wall)
 *  kind 1 (OS-NT step):   slot(i, r) = i Npad + a       (a >= 0),  inv(i) Npad + h (wall)
 * out: host int32 [R][18] (run-major, as the device holds them without the
 * padding words), entry i - 1 of row r for i = 1..18.  *available is set to 1
 * when the lattice has the tables, else 0 (pressure markers, or a grid of
 * 2^31 slots or more: the steps then decode run_adj) and out is left alone.
 * out may be NULL to ask for availability only. */
LBM_API int lbm_export_run_slots(lbm_lattice* lat, int kind, int32_t* out, int* available);

/* Adjacency entries of chosen nodes only (lattices too large to export in
 * full).  nodes: host int64 [count] in [0, N); out: host int32 [18][count]. */
LBM_API int lbm_export_adjacency_rows(const lbm_lattice* lat, const int64_t* nodes, int64_t count, int32_t* out);

/* LBM_OK if the `count` doubles at device address `values` (e.g. the sums of
 * lbm_macroscopic) are all finite, LBM_ERR_NONFINITE otherwise.  Synchronises
 * `stream` to read them; a guard between steps, not for the timed loop. */
LBM_API int lbm_check_finite(const double* values, int64_t count, void* stream);

/* Host image of the FP64 step's moment arithmetic, so that it can be tested
 * without a GPU.  The LBM_F64 step kernels form a node's moments -- the
 * density deviation sum_i d_i, the momentum sum_i c_i d_i, and the pair sums
 * and differences d_a +- d_inv(a) that the TRT collision (Sect. 2) splits
 * into even and odd parts -- as exact fixed-point sums on the integer pipe,
 * each rounded once to the nearest double; this runs the same routine on the
 * host.  d: host double [n][19] (node-major, direction order as above);
 * out: host double [n][22]: drho, jx, jy, jz, sa_1..sa_9, da_1..da_9, pair k
 * holding directions 2k-1 and 2k.  A PDF more than 5 binades below the node's
 * largest loses the bits below 2^-57 of that largest (truncated).  A node
 * with an Inf or NaN PDF, or one of magnitude >= 2^1017, gets drho = NaN.
 * LBM_ERR_ARG for NULL pointers or n < 0. */
LBM_API int lbm_exact_moments_host(const double* d, int64_t n, double* out);

/* Host image of the FP64 step's fixed-point pair update, so that it can be
 * tested without a GPU.  The TRT collision (Sect. 2) relaxes the even and odd
 * parts of each opposite pair (a, b = inv a); with the node's velocity u and
 * the axis-class terms K0, T, O (halved for the face diagonals) the pair
 * becomes p_a,b = e +- o, e = K0 + (c_a.u)(c_a.T) + qp (d_a + d_b),
 * o = qm (d_a - d_b) + c_a.O, qm = (1 - l-)/2, qp = (1 - l+)/2.  The LBM_F64
 * step kernels evaluate this in 64-bit fixed point at a scale 2^(es - 1080)
 * tied to the node's largest PDF, with one rounding to double per output,
 * whenever the node's values lie in that scale's range; this runs the same
 * routine on the host.  d: host double [n][19] (node-major); terms: host
 * double [n][10]: ux, uy, uz, K0, Tx, Ty, Tz, Ox, Oy, Oz; flags: bit 0 for
 * the l+ = 1 form (qp must be 0), bit 1 to take the general conversions
 * everywhere (the kernels take shorter ones for positive values in a common
 * range; the results are the same bits).  out: host double [n][19]: out[0] = es, out[1..18]
 * the post-collision pair values; ok: host int [n], 0 where the node is
 * outside the range (out is then 0; the kernels take the FP64 update there).
 * Each value is within 8 units of 2^(es - 1080) of the exact rational result,
 * before its rounding to nearest.  LBM_ERR_ARG for NULL pointers, n < 0, or
 * |qm| or |qp| >= 1/2. */
LBM_API int lbm_fx_pairs_host(const double* d, const double* terms, int64_t n, double qm, double qp, int flags,
                              double* out, int* ok);

/* Check the host tables: entries in range, adjacency reciprocity
 * (adj[i][n] = m >= 0  <=>  adj[inv i][m] = n), run table decoding back to the
 * adjacency list exactly, runs sorted and covering [0, N).  Returns
 * LBM_ERR_TABLE with a message naming the first violation. */
LBM_API int lbm_validate_tables(const lbm_lattice* lat);

/* ---- device tables -------------------------------------------------------------- */

/* Bytes of the caller-owned device buffer that holds the tables selected by
 * `which` (LBM_TABLES_ADJ | LBM_TABLES_RIA). */
LBM_API int lbm_device_table_bytes(const lbm_lattice* lat, int which, size_t* bytes);

/* Copy the selected tables into dev_tables (device, >= lbm_device_table_bytes,
 * 256-byte aligned) on `stream` and remember the device addresses in the
 * handle.  The buffer must outlive every later device call on the handle.
 * The host source of the copy is the handle itself, so the handle must not be
 * freed before the copy completes. */
LBM_API int lbm_lattice_upload(lbm_lattice* lat, int which, void* dev_tables, size_t bytes, void* stream);

/* Bytes of one PDF grid (19 * Npad elements) of a precision. */
LBM_API int lbm_pdf_bytes(const lbm_lattice* lat, int prec, size_t* bytes);

/* ---- state set-up and read-back ------------------------------------------------ */

/* Fill a grid with the equilibrium state f^eq(rho0, u0) at every node, stored
 * in `layout` (the state whose canonical form is f^eq).  pdf: device grid. */
LBM_API int lbm_init_equilibrium(const lbm_lattice* lat, int prec, const lbm_params* params, void* pdf,
                         int layout, double rho0, const double u0[3], void* stream);

/* Store a canonical FP64 state F (device [19][N]) into a grid of `layout`
 * (rounded to the storage precision). */
LBM_API int lbm_load_canonical(const lbm_lattice* lat, int prec, const lbm_params* params, const double* F,
                       void* pdf, int layout, void* stream);

/* Gather the canonical FP64 state F (device [19][N]) of a grid. */
LBM_API int lbm_canonical_pdfs(const lbm_lattice* lat, int prec, const lbm_params* params, const void* pdf,
                       int layout, double* F, void* stream);

/* ---- the stream-collide step --------------------------------------------------- */

/* One OS-NT step (Sect. 4, "Loop Balance"): every node pulls its 19 PDFs from
 * the neighbours in `src` (indirectly, through the adjacency list or the RIA
 * runs), collides them with the TRT operator (Sect. 2) with body force g and
 * optional Brinkman drag s, and stores the result at its own slots in `dst`
 * with streaming (evict-first) stores.  src, dst: device grids in the
 * LBM_LAYOUT_OSNT layout, distinct.  s: device float [N] in [0, 1] or NULL.
 * ria = 0 uses the adjacency list (OS-NT, B_l = 38p + 72 B/FLUP), 1 the RIA
 * table (OS-NT-R, Sect. 4.1); the matching table must have been uploaded. */
LBM_API int lbm_step_osnt(const lbm_lattice* lat, int prec, const lbm_params* params, const void* src,
                  void* dst, const float* s, int ria, void* stream);

/* One AA-pattern step on the single grid `pdf` (Sect. 4, "Loop Balance",
 * AA pattern).  parity 0 (even step): read the 19 local PDFs, collide, write
 * them to the opposite local slots (direct addressing only).  parity 1 (odd
 * step): read the neighbours' opposite slots, collide, write back to the same
 * slots (indirect).  The grid must be in layout AA_EVEN before an even step
 * and AA_ODD before an odd one.  ria selects the odd step's addressing as in
 * lbm_step_osnt (AA-R, Sect. 4.1). */
LBM_API int lbm_step_aa(const lbm_lattice* lat, int prec, const lbm_params* params, void* pdf, int parity,
                const float* s, int ria, void* stream);

/* `steps` consecutive AA steps starting with parity start_parity. */
LBM_API int lbm_run_aa(const lbm_lattice* lat, int prec, const lbm_params* params, void* pdf,
               int start_parity, int steps, const float* s, int ria, void* stream);

/* ---- Esoteric Twist: the third single-grid form (named in Sect. 1 and Sect. 4) ----
 * The paper lists Geier's Esoteric Twist with OS-NT and the AA pattern as the
 * lowest-loop-balance propagation schemes but does not evaluate it.  Layout
 * used here: the link between node n and n + c_i keeps its two slots at
 * location n + max(c_i, 0), so every step touches the node itself and the six
 * locations +x, +y, +z, +x+y, +x+z, +y+z.  Even step: node n reads f_i from
 * slot i at n + max(-c_i, 0) and writes P_j to slot inv(j) at n + max(c_j, 0);
 * odd step: slots inv(i) and j.  A link to a wall or a pressure face writes the
 * bounced value (P_j, or 2 w rho_bc - P_j) into the pair's other slot, which
 * the node reads next.  Locations that are not fluid nodes but hold slots get
 * "phantom" storage indices N .. S-1, ordered lexicographically (x fastest) by
 * their coordinates (wrapped on periodic axes; up to X, Y, Z on the far faces).
 * Tables: 6 int32 locations and one uint32 link mask per node, so
 * B_l = 38p + 28 B/FLUP on every step.  Grid: [19][Spad] of the precision's
 * element type. */

/* Esoteric Twist sizes, deriving its tables on first use: S = N + phantom
 * locations, Spad = the grid stride (S rounded up to 128), and optionally the
 * phantoms' coordinates (host int32 [S-N][3], x y z).  LBM_ERR_UNSUPPORTED for
 * a partition's local lattice, or a lattice without node coordinates that
 * needs phantoms. */
LBM_API int lbm_et_info(lbm_lattice* lat, int64_t* S, int64_t* Spad, int32_t* phantom_xyz);

/* The Esoteric Twist tables on the host (bit-exact comparison): nb (int32
 * [6][N]) the storage index of n + (+x, +y, +z, +x+y, +x+z, +y+z); mask (uint32
 * [N]) bit i-1 set when the pull of direction i at n meets a marker, bit
 * 18 + r when that marker is a pressure face, r the rank of i among the ten
 * directions with c_ix != 0 (1, 2, 7, ..., 14).  Either may be NULL. */
LBM_API int lbm_export_et_tables(lbm_lattice* lat, int32_t* nb, uint32_t* mask);

/* The run-length coding of the Esoteric Twist tables (the RIA idea of
 * Sect. 4.1 applied to them): node n continues the run of n-1 when its six
 * locations are n-1's plus one and the masks are equal.  R (host) = number of
 * runs; run_start (int32 [R+1]) the first node of each run and N; run_nb
 * (int32 [6][R]) and run_mask (uint32 [R]) the entries of each run's first
 * node.  Any pointer may be NULL (ask for R first). */
LBM_API int lbm_export_et_runs(lbm_lattice* lat, int64_t* R, int32_t* run_start, int32_t* run_nb,
                               uint32_t* run_mask);

/* One Esoteric Twist step of the grid `pdf` ([19][Spad], layout ET_EVEN before
 * a parity-0 step, ET_ODD before a parity-1 one), in place.  Needs the
 * LBM_TABLES_ET tables uploaded.  s: Brinkman field or NULL.  ria = 0 reads
 * the plain tables (28 B per node and step); ria = 1 their run table (ET-R:
 * about 28 r B, r = runs per node). */
LBM_API int lbm_step_et(const lbm_lattice* lat, int prec, const lbm_params* params, void* pdf, int parity,
                        const float* s, int ria, void* stream);

/* `steps` consecutive Esoteric Twist steps starting with parity start_parity. */
LBM_API int lbm_run_et(const lbm_lattice* lat, int prec, const lbm_params* params, void* pdf, int start_parity,
                       int steps, const float* s, int ria, void* stream);

/* ---- macroscopic quantities and reductions ------------------------------------- */

/* Bytes of the device workspace the reductions below need (per-block FP64
 * partial sums). */
LBM_API int lbm_reduce_workspace_bytes(const lbm_lattice* lat, size_t* bytes);

/* Density and velocity of every node and FP64 global sums.  The velocity is
 * the force-corrected u = (j0/rho + g/2)/(1 + s/2).  rho (device double [N]),
 * u (device double [3][N]) and sums (device double [4]: sum rho, sum rho u_x,
 * sum rho u_y, sum rho u_z) may each be NULL.  workspace: device, at least
 * lbm_reduce_workspace_bytes.  Sums are deterministic (fixed reduction order).
 * No counterpart in the paper beyond the LBM moments of Sect. 2. */
LBM_API int lbm_macroscopic(const lbm_lattice* lat, int prec, const lbm_params* params, const void* pdf,
                    int layout, const float* s, double* rho, double* u, double* sums,
                    void* workspace, size_t ws_bytes, void* stream);

/* lbm_macroscopic for callers that cannot allocate device memory.  No
 * counterpart in the paper: it exists because lbm_macroscopic needs a
 * caller-provided workspace, and some callers cannot get one (a host
 * application whose pool allocator owns all device memory, or a loop in which
 * a possibly synchronising cudaMalloc is not allowed).  Same arguments and
 * results as lbm_macroscopic without the workspace: the per-block partial
 * sums live in a fixed 4 MiB array inside the library (present on every GPU
 * that loads it, until unload), so at most 16,777,216 fluid nodes are
 * accepted (LBM_ERR_ARG otherwise).  Every layout of lbm_macroscopic is
 * accepted, with the same table requirements.  The first call on a device
 * looks up that array's address with the device current and caches it; make
 * it before any stream capture, and do not call this entry point across a
 * cudaDeviceReset (the cached address would be stale).  All calls share the
 * array: calls whose kernels overlap on the GPU race and may return wrong
 * sums.  Allocates nothing. */
LBM_API int lbm_macroscopic_noalloc(const lbm_lattice* lat, int prec, const lbm_params* params, const void* pdf,
                                    int layout, const float* s, double* rho, double* u, double* sums,
                                    void* stream);

/* ---- pattern-specific bandwidth kernels ---------------------------------------- */
/* The GPU counterparts of the paper's micro-benchmarks (Sect. 5.2, Table 3),
 * which give the bandwidth b of the roofline P = b / B_l for each access
 * pattern.  kind 0 (CNT-kA): copy `arrays` arrays of bytes_per_array bytes from
 * src to dst with streaming stores (the OS-NT pattern); kind 1 (U-kA): update
 * the arrays of dst in place (the AA even-step pattern; src unused).  The
 * arrays are consecutive slices of each buffer.  bytes_per_array: a positive
 * multiple of 16; buffers 16-byte aligned.  One launch, asynchronous. */
LBM_API int lbm_bandwidth_kernel(int kind, const void* src, void* dst, int64_t bytes_per_array, int arrays,
                                 void* stream);

/* The FP64 pipe's throughput, the compute roof beside the bandwidth roof of
 * Sect. 5.2 for the native FP64 step (whose arithmetic, not HBM, bounds it on
 * this GPU).  One launch of `threads` threads (a positive multiple of 256, at
 * most 2^31), each running 8 independent chains of `iters` fused
 * multiply-adds x <- fma(x, 1, 1) (8 * threads * iters DFMA in total).  out:
 * device double [threads]; out[t] = 8 (t mod 1024) + 28 + 8 iters exactly.
 * iters in [1, 2^24].  Asynchronous on `stream`. */
LBM_API int lbm_fp64_peak_kernel(double* out, int64_t threads, int iters, void* stream);

/* ---- objective, discrete adjoint and checkpointed gradient ------------------------ */
/* None of these has a counterpart in the paper: they differentiate the step of
 * Eq. 1 (TRT collision, Sect. 2; pull streaming, Sect. 4) with respect to the
 * per-node Brinkman solid fraction s.  The adjoint arrays ("lambda") have the
 * grid layout [19][Npad] and element type double for LBM_F64 / LBM_F64_DF,
 * float for LBM_F32 and LBM_F16S (the adjoint step itself always runs in the
 * element type's native arithmetic). */

/* Mean x-momentum objective J = (1/N) sum_n rho_n u_x,n of the canonical state
 * of `pdf` (compensated FP64 sum) written to J (device double[1]).  Optional
 * outputs: lambda_T = dJ/dF (adjoint layout) and grad_s (device double [N],
 * overwritten) = the direct term dJ/ds.  workspace as for lbm_macroscopic. */
LBM_API int lbm_objective_flux(const lbm_lattice* lat, int prec, const lbm_params* params, const void* pdf,
                               int layout, const float* s, double* J, void* lambda_T, double* grad_s,
                               void* workspace, size_t ws_bytes, void* stream);

/* One discrete-adjoint step: given the OS-NT grid G_n of step n (its pull
 * gather is the canonical state F_n) and lambda_next = dJ/dF_{n+1}, write
 * lambda_n = dJ/dF_n and add (dF_{n+1}/ds)^T lambda_next to grad_s (device
 * double [N], accumulated; may be NULL).  s may be NULL (s = 0).  lambda_next
 * and lambda_n must not overlap.  ria selects the addressing as for the step. */
LBM_API int lbm_adjoint_step(const lbm_lattice* lat, int prec, const lbm_params* params, const void* G_n,
                             const void* lambda_next, void* lambda_n, const float* s, double* grad_s, int ria,
                             void* stream);

/* Device workspace of the checkpointed gradient: ceil(T/K) checkpoint grids,
 * the final grid, max(2, K-1) recompute grids, two adjoint grids and the
 * reduction partials. */
LBM_API int lbm_ckpt_workspace_bytes(const lbm_lattice* lat, int prec, int T, int K, size_t* bytes);

/* Forward pass of J(s) after T OS-NT steps from the OS-NT grid G0 (not
 * modified), storing a checkpoint every K steps in the workspace; J written to
 * device double[1].  K ~ sqrt(T) balances memory and recomputation. */
LBM_API int lbm_flux_forward(const lbm_lattice* lat, int prec, const lbm_params* params, const void* G0,
                             const float* s, int T, int K, int ria, void* workspace, size_t ws_bytes, double* J,
                             void* stream);

/* Backward pass after lbm_flux_forward with the same arguments and
 * workspace: segment by segment in reverse, recompute the K states from the
 * checkpoint, then run the adjoint steps back through them.  grad_s (device
 * double [N]) is overwritten with dJ/ds; lambda_0 (adjoint layout, may be
 * NULL) receives dJ/dF_0. */
LBM_API int lbm_flux_backward(const lbm_lattice* lat, int prec, const lbm_params* params, const float* s, int T,
                              int K, int ria, void* workspace, size_t ws_bytes, double* grad_s, void* lambda_0,
                              void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_H */
