/*
 * mk.h -- C ABI of libmk: exhaustive evaluation of modal formulas over every
 * labelled Kripke frame up to n worlds, on one GB300 GPU (sm_103a).
 *
 * Conventions for every call
 *   - Return value: 0 (MK_OK) on success, a negative MK_E_* code otherwise;
 *     mk_strerror() gives its text.  A call that fails leaves its outputs
 *     undefined and launches nothing after the failing step.
 *   - Pointers named d_* are device pointers (any allocator; the Python
 *     binding uses PyTorch).  Pointers named h_* (and all other pointers) are
 *     host pointers.  The caller owns every buffer; the library allocates no
 *     device memory: scratch comes from a caller-provided workspace of the size
 *     the matching *_workspace_size() call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device calls are asynchronous on it; outputs are valid once
 *     the stream has been synchronised.
 *   - Device-side failures (a malformed program, a limit exceeded inside a
 *     kernel, an iteration limit reached) are OR-ed as MK_ST_* bits into the
 *     caller's int32 device word d_status (clear it before the call);
 *     mk_status_error() maps a read-back status to an MK_E_* code.
 *   - Calls on distinct buffers and streams are thread-safe.  The library's
 *     only global state is a mutex-guarded cache of the kernel attributes it
 *     has set on each device (and the fixed scratch of mk_census_noalloc).
 *
 * Encodings (readings of the paper where it leaves them open)
 *   - World w of an n-world frame is bit w of a mask; full = 2^n - 1 (Sec. 3).
 *   - Frame (K) index f: R(w,v) holds iff bit w*n+v of f is set, so the
 *     successor mask succ[w] is bits [w*n, w*n+n) of f.
 *   - Valuation index x: p_i holds at w iff bit i*n+w of x is set.
 *   - k = 1 + the highest variable index in the formula (0 if none).
 *   - A layer's valuations are exhaustive (x = 0 .. 2^(k n)-1) when S == 0,
 *     k <= 1 or 2^(k n) <= S; otherwise the S sampled values of that layer
 *     (their low k*n bits), in slot order, counted with multiplicity.
 */
#ifndef MK_H
#define MK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- limits */
#define MK_MAX_NODES 64          /* |phi| of a compiled formula               */
#define MK_MAX_CODE 96           /* instructions per program (<= nodes + pushes) */
#define MK_MAX_STACK 4           /* saved truth sets per program               */
#define MK_MAX_VARS 4            /* p0..p3 (paper's limit, Sec. 11)            */
#define MK_MAX_WORLDS_EXH 6      /* exhaustive frames: K index < 2^36          */
#define MK_MAX_WORLDS_SAMPLED 8  /* sampled separation frames                  */
#define MK_MAX_CERT_WORLDS 32    /* certificates (u32 successor masks)         */

/* ----------------------------------------------------------- error codes */
#define MK_OK 0
#define MK_E_SYNTAX (-1)     /* formula text does not parse                   */
#define MK_E_TOO_LONG (-2)   /* more than MK_MAX_NODES nodes / MK_MAX_CODE ops */
#define MK_E_VARS (-3)       /* variable index >= MK_MAX_VARS                 */
#define MK_E_SLOTS (-4)      /* needs more than MK_MAX_STACK stack entries     */
#define MK_E_ARG (-5)        /* invalid argument or configuration             */
#define MK_E_WORKSPACE (-6)  /* workspace missing or too small                */
#define MK_E_CUDA (-7)       /* a CUDA runtime call failed                    */
#define MK_E_PROGRAM (-8)    /* device saw a malformed program                */
#define MK_E_LIMIT (-9)      /* a size limit was exceeded (e.g. k*n)          */
#define MK_E_INTERNAL (-10)  /* internal consistency check failed             */
#define MK_E_TIMEOUT (-11)   /* a bounded device wait ran out                 */

/* device status bits (OR-ed into *d_status) */
#define MK_ST_PROGRAM 1u     /* malformed program: its results are not valid  */
#define MK_ST_LIMIT 2u       /* exhaustive valuations with k*n > 24           */
#define MK_ST_INTERNAL 4u    /* class-table size mismatch or similar          */
#define MK_ST_TIMEOUT 8u     /* a bounded wait gave up                        */
#define MK_ST_INDEX 16u      /* an index read from device memory was out of  */
                             /* range (the entry is skipped)                   */

/* ----------------------------------------------------- frame classes */
#define MK_CLASS_K 1u        /* all frames                                    */
#define MK_CLASS_T 2u        /* reflexive                                     */
#define MK_CLASS_S4 4u       /* reflexive and transitive (preorders)          */
#define MK_CLASS_S5 8u       /* equivalence relations                         */
#define MK_CLASS_K4 16u      /* transitive (the frames of K4; not in the      */
                             /* uneven path, whose jobs are K, T, S4 or S5)    */

/* --------------------------------------------------- compiled programs */
/* A program is postfix code for an accumulator machine over truth sets (the
   recurrence of Thm. 1): A is the current truth set (one n-world set per
   register word lane), st[0..MK_MAX_STACK) a small stack of saved sets.
   Instruction byte = op | operand << 5 (op < MK_NUM_OPS, operand < 8); the
   operand is a variable index i or a stack depth d:
     LDV i   A = [[p_i]]            LDT  A = W              LDF  A = {}
     NOT     A = W \ A              BOX  A = {w : succ[w] subset of A}
     DIA     A = {w : succ[w] meets A}          (Lemma 1, eqs. box/dia)
     PUSH d  st[d] = A
     AND_S d / OR_S d / IFF_S d   A = st[d] op A
     IMP_S d  A = st[d] -> A      RIMP_S d  A = A -> st[d]
     AND_V i / OR_V i             A = A op [[p_i]]
     IMP_V i  A = A -> [[p_i]]    RIMP_V i  A = [[p_i]] -> A
     LDNV i  A = W \ [[p_i]]
     AND_NV i / OR_NV i           A = A op (W \ [[p_i]])
     IMP_NV i A = A -> (W \ [[p_i]])
     BOX_V i / DIA_V i            A = box / dia of [[p_i]]
     BOX_NV i / DIA_NV i          A = box / dia of W \ [[p_i]]
   A program ends with the formula's truth set in A.  The compiler emits
   negation normal form (negations pushed to the atoms by De Morgan and the
   duality of box and diamond), so NOT appears only above a biconditional. */
enum {
    MK_OP_LDV = 0, MK_OP_LDT = 1, MK_OP_LDF = 2, MK_OP_NOT = 3, MK_OP_BOX = 4, MK_OP_DIA = 5,
    MK_OP_PUSH = 6, MK_OP_AND_S = 7, MK_OP_OR_S = 8, MK_OP_IMP_S = 9, MK_OP_RIMP_S = 10,
    MK_OP_IFF_S = 11, MK_OP_AND_V = 12, MK_OP_OR_V = 13, MK_OP_IMP_V = 14, MK_OP_RIMP_V = 15,
    MK_OP_LDNV = 16, MK_OP_AND_NV = 17, MK_OP_OR_NV = 18, MK_OP_IMP_NV = 19,
    MK_OP_BOX_V = 20, MK_OP_DIA_V = 21, MK_OP_BOX_NV = 22, MK_OP_DIA_NV = 23,
    MK_NUM_OPS = 24
};

typedef struct {
    uint16_t nodes;        /* |phi|: node count of the source text          */
    uint8_t n_instr;       /* instructions in code[]                        */
    uint8_t nvars;         /* k                                             */
    uint8_t modal_depth;   /* nesting depth of []/<> in the source          */
    uint8_t depth;         /* stack entries used (<= MK_MAX_STACK)          */
    uint8_t n_modal;       /* box / diamond steps                           */
    uint8_t n_bool;        /* negating and binary instructions              */
    uint8_t code[MK_MAX_CODE];
} mk_program;              /* 104 bytes, plain data                         */

/* Compile formula text to a program (host).  Grammar: atoms p0..p3 (p, q, r,
   s = p0..p3), T, F; unary ~ ! not [] box <> dia; binary & and, | or, ->
   (right associative), tightest first; parentheses.  Constant subformulas are
   folded (e.g. []T = T, <>F = F), which leaves every truth set unchanged.
   *err_pos (may be NULL) receives the byte offset of a syntax error.
   Formula grammar and node count: Sec. 2; postfix programs: Sec. 4. */
int mk_compile(const char *text, mk_program *out, int32_t *err_pos);

/* Compile "phi <-> psi" into one program whose truth set is the set of
   worlds where phi and psi agree (the biconditional of Prop. 4). */
int mk_compile_iff(const char *phi, const char *psi, mk_program *out, int32_t *err_pos);

/* ----------------------------------------------------------- the census */
typedef struct {
    uint16_t block;        /* threads per CTA: 128, 256 or 512 (0 = 256)    */
    uint16_t tile;         /* formulas per CTA, 1..64 (0 = 16)              */
    uint16_t units;        /* units per dispatched instruction: valuations  */
                           /* (census: 2, 4 or 8; 0 = 8) -- the same program */
                           /* step is applied to that many units at once      */
    uint16_t persistent;   /* 1 = one persistent launch over a work queue   */
} mk_tune;

typedef struct {
    uint32_t classes;          /* MK_CLASS_* bits                                */
    uint8_t n_min, n_max;      /* 1 <= n_min <= n_max <= 6                       */
    uint8_t max_depth;         /* largest program depth in the batch (0 = the    */
                               /* limit MK_MAX_STACK); sizes the device stack;   */
                               /* a deeper program sets MK_ST_PROGRAM            */
    uint8_t max_vars;          /* largest variable count in the batch (0 =       */
                               /* unknown); only caps the valuation split below  */
    uint32_t samples;          /* S (0 = always exhaustive)                      */
    uint32_t vsplit;           /* valuation chunks per layer, <= 4096: 0 = auto  */
                               /* (split a layer whose grid of frame words x     */
                               /* formula tiles is under 1,216 CTAs, four waves  */
                               /* of 2 CTAs on 152 SMs), 1 = never, v > 1 = v    */
                               /* chunks on every layer.  Only the default tune  */
                               /* (units 8, block 256) splits.  Results are the  */
                               /* same either way; a split layer needs the       */
                               /* workspace's frame-word bitmap (below)          */
    const uint32_t *d_samples; /* device [(n_max+1) * S]: row n = layer n's S    */
                               /* sampled valuations; NULL iff S == 0            */
    uint64_t frame_lo;         /* only frames with K index in [frame_lo,         */
    uint64_t frame_hi;         /*  frame_hi); 0, UINT64_MAX = all                */
    mk_tune tune;              /* zeros = defaults                               */
} mk_census_cfg;

typedef struct {
    uint64_t cm_count;         /* refuted (frame, valuation) pairs               */
    uint64_t frames_refuted;   /* frames with at least one refuted valuation     */
    uint64_t witness_key;      /* least (frame, valuation, world), packed as     */
                               /* f << 27 | x << 3 | w (x: valuation index or    */
                               /* sample slot); UINT64_MAX = no countermodel     */
} mk_result;

/* Workspace bytes mk_census needs for this configuration and batch: the
   S4/S5/K4 frame lists and, when some layer splits its valuations, a bitmap of
   nprog x (that layer's frame words) u32 words in which the chunks OR their
   refuted frames, plus one u32 counter per formula tile (the last CTA of a
   tile to finish counts the bitmap).  Given less (but at least the lists'
   share), mk_census runs every layer unsplit. */
size_t mk_census_workspace_size(const mk_census_cfg *cfg, int32_t nprog);

/* Census (Alg. 1 over every selected (class, n) layer, Thm. 2): for each
   program p, each selected class c (in the order K, T, S4, S5, K4) and each
   n in [n_min, n_max], writes
       d_out[(p * ncls + c) * (n_max - n_min + 1) + (n - n_min)]
   where ncls = number of selected classes.  d_progs: device [nprog]
   programs from mk_compile.  The refuted flag is cm_count > 0; the minimal
   countermodel size is the least n with cm_count > 0. */
int mk_census(const mk_program *d_progs, int32_t nprog, const mk_census_cfg *cfg,
              mk_result *d_out, int32_t *d_status, void *d_workspace, size_t ws_bytes,
              void *stream);

/* The census without a caller-provided workspace, for callers that cannot
   allocate device memory: a C program or language binding that only passes
   pointers it already owns, or code that must not call cudaMalloc/cudaFree
   because they synchronise the device.  The paper has no counterpart; it
   is a packaging of mk_census.  Arguments and results are those of
   mk_census; the scratch space is a fixed array of MK_NOALLOC_SCRATCH_BYTES
   inside the library, held on every GPU that loads it until the process
   exits.  Configurations whose S4/S5/K4 frame lists exceed that limit (S4 or
   S5 at n = 6, K4 at n >= 5) are rejected with MK_E_WORKSPACE before anything is
   launched; layers split their valuations only when the split bitmap also
   fits (mk_census_workspace_size <= the limit).  Every call made outside
   stream capture looks up the array's address on the current device
   (cudaGetSymbolAddress, which allocates nothing) and remembers it; a call
   made while its stream is being captured uses the address remembered for
   that device, or looks it up if there is none.  So a device reset
   (cudaDeviceReset, or the primary context torn down and re-created)
   between calls is harmless, but after one make an uncaptured call before
   capturing, and make the first call on a device before any stream
   capture.  All calls share the one array, and it keeps
   the last call's contents: every part of it that a call reads is written
   by that call first, but calls whose work overlaps on the GPU (different
   streams, or different host threads) race on it, so serialise them.
   Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define MK_NOALLOC_SCRATCH_BYTES (1u << 20)
int mk_census_noalloc(const mk_program *d_progs, int32_t nprog, const mk_census_cfg *cfg,
                      mk_result *d_out, int32_t *d_status, void *stream);

/* ------------------------------------------------------ uneven batches */
/* Formulas of very different lengths, each with its own class and n_max,
   evaluated in ONE persistent launch that takes work items from a queue
   (Sec. 8 measures fused vs separate launches; here the fusion spans
   classes, sizes and lengths).  The host builds a plan (mk_plan_uneven):
   for every layer (class c, n) the jobs with that class and n_max >= n are
   sorted by cost, cut into tiles of formulas of similar length, and every
   tile is split into items of a few thousand frame words; items are
   ordered longest first.  The caller copies the plan to device memory as
   is; mk_census_uneven then clears the outputs, builds the S4/S5 lists,
   resets the queue cursor and runs the persistent kernel -- all stream
   operations, so the whole call can be captured in a CUDA graph (after one
   uncaptured call, which sets kernel attributes). */
typedef struct {
    int32_t prog;          /* index into the program array                  */
    uint8_t cls;           /* 0 K, 1 T, 2 S4, 3 S5                           */
    uint8_t n_max;         /* layers n = 1..n_max, n_max <= 6                */
    uint16_t reserved;
} mk_job;

typedef struct {
    uint32_t lbeg;         /* first entry of the tile in the plan's job list */
    uint16_t np;           /* jobs in the tile                               */
    uint8_t n;             /* worlds                                         */
    uint8_t cls;           /* 0 K, 1 T, 2 S4, 3 S5                           */
    uint64_t w0, w1;       /* frame words [w0, w1) of the layer (32 frames   */
                           /* per word, in class order)                      */
} mk_work_item;            /* 24 bytes                                       */

typedef struct {
    uint64_t bytes;        /* plan size                                      */
    uint32_t nitems;       /* work items                                     */
    uint32_t nlist;        /* entries of the job list (one per job and n)    */
    uint32_t list_off;     /* byte offset of the job list (uint32 job ids)   */
    uint32_t items_off;    /* byte offset of the items (mk_work_item)        */
    uint8_t n_max;         /* largest n over the jobs                        */
    uint8_t max_depth;     /* largest program depth                          */
    uint16_t block;        /* threads per CTA the plan was cut for           */
    uint16_t units;        /* valuations per dispatched instruction          */
    uint16_t tile_cap;     /* largest tile (formulas per work item)          */
    double ops;            /* estimated logic ops of the batch               */
} mk_plan_info;

/* Build a plan (host).  tiles[4]: formulas per tile for programs of <= 8,
   <= 16, <= 32 and more instructions (NULL: 16 each); tune: block and
   units (zeros: 256 and 8).  h_plan == NULL only fills *info (size).
   Returns MK_E_WORKSPACE if plan_bytes < info->bytes. */
int mk_plan_uneven(const mk_program *h_progs, int32_t nprog, const mk_job *h_jobs, int32_t njobs,
                   uint32_t samples, const uint16_t *tiles, const mk_tune *tune, void *h_plan,
                   size_t plan_bytes, mk_plan_info *info);

size_t mk_uneven_workspace_size(const mk_plan_info *info);

/* Run the plan: for every job j and n <= its n_max, writes
   d_out[j * 6 + (n - 1)] (results of the job's class on n worlds); entries
   for n > n_max are left cleared (cm_count 0, no witness).  d_plan: the
   plan bytes in device memory; d_samples: [(n_max+1) * S] as in the census. */
int mk_census_uneven(const mk_program *d_progs, const mk_job *d_jobs, int32_t njobs, const void *d_plan,
                     const mk_plan_info *info, uint32_t samples, const uint32_t *d_samples,
                     mk_result *d_out, int32_t *d_status, void *d_workspace, size_t ws_bytes,
                     void *stream);

/* Number of class-c frames on n worlds that mk_census enumerates (K: 2^(n^2),
   T: 2^(n^2-n), S4: preorders, S5: equivalence relations, K4: transitive
   relations); 0 if n > 6. */
uint64_t mk_class_frames(uint32_t cls, int32_t n);

/* ------------------------------------------------------- certificates */
typedef struct {
    const char *phi;           /* formula text                                   */
    const char *psi;           /* NULL: countermodel certificate for phi;        */
                               /* else: a world where phi and psi disagree       */
    uint8_t n;                 /* worlds, 1..32                                  */
    uint8_t cls;               /* 0 K, 1 T, 2 S4, 3 S5, 4 K4: the frame must be  */
                               /* in it                                          */
    uint8_t world;             /* the pointed world                              */
    uint8_t reserved;
    uint32_t succ[MK_MAX_CERT_WORLDS];  /* successor masks                       */
    uint32_t val[MK_MAX_VARS];          /* variable masks                        */
} mk_cert;

/* Certificate check (Def. 1, Prop. 2), host only: its own parser and a
   recursive evaluator over explicit successor sets, sharing no code with the
   compiler or the kernels.  Returns 1 if valid (frame in class, and phi false
   at world -- or phi and psi differ there), 0 if not, < 0 if malformed. */
int mk_certify(const mk_cert *c);

/* Decode a census witness key of program h_prog (host copy) on the class-cls,
   n-world layer into a certificate (phi text supplied by the caller).
   h_samples_n: the layer's S sampled valuations (host), NULL iff S == 0. */
int mk_witness_cert(const mk_program *h_prog, const char *phi, uint32_t cls, int32_t n,
                    uint32_t samples, const uint32_t *h_samples_n, uint64_t key,
                    mk_cert *out);

/* ------------------------------------------------------- separation */
typedef struct {
    uint8_t n_exh_min, n_exh_max;  /* exhaustive K sizes scanned, 1..6          */
    uint8_t n_smp_min, n_smp_max;  /* sampled sizes, 7..8 (0, 0 = none)         */
    uint32_t samples;              /* valuation samples S (as in the census)    */
    const uint32_t *d_samples;     /* device [(8+1) * S] or NULL iff S == 0     */
    uint64_t frames_per_n;         /* sampled relations per sampled size        */
    uint64_t seed;                 /* seed of the relation stream               */
    uint64_t frame_lo, frame_hi;   /* K-index range of exhaustive sizes         */
    mk_tune tune;
    uint8_t max_depth;             /* largest program depth among phi and psi   */
                                   /* (0 = MK_MAX_STACK); a deeper program sets */
                                   /* MK_ST_PROGRAM and its pair is skipped      */
} mk_separate_cfg;

/* Distinguishing-pair search (Def. 2, Prop. 4): for each pair i, the least
   (n, frame, valuation, world) at which phi_i and psi_i take different
   truth values, over the K frames of n_exh_min..n_exh_max worlds in K-index
   order, then the sampled relations of n_smp_min..n_smp_max worlds in sample
   order (sizes are searched in that order; a pair with a split at one size is
   not searched at later sizes).  Writes d_split[i] = the packed key
       sampled << 63 | (n - 1) << 60 | f << 24 | x << 3 | w
   (f: K index or sample number < 2^36; x < 2^21; w < 8), UINT64_MAX if the
   pair agrees everywhere searched.  Relations of sampled sizes come from
   mk_sample_relation(seed, n, s).  The workspace (mk_separate_workspace_size
   bytes, 16-byte aligned, contents need not be initialised; MK_E_WORKSPACE
   if smaller) holds the list of pairs still unsplit, rebuilt on the device
   before every launch so that only those pairs are staged. */
size_t mk_separate_workspace_size(const mk_separate_cfg *cfg, int32_t npairs);
/* Kernel launches one mk_separate call with this configuration issues (the
   keys' initialisation, then an active-pair list and a search per chunk);
   -1 for an invalid configuration. */
int64_t mk_separate_launches(const mk_separate_cfg *cfg, int32_t npairs);
int mk_separate(const mk_program *d_phi, const mk_program *d_psi, int32_t npairs,
                const mk_separate_cfg *cfg, uint64_t *d_split, int32_t *d_status,
                void *d_workspace, size_t ws_bytes, void *stream);

/* The row-major edge mask of sampled relation s on n <= 8 worlds: nine
   SplitMix64 draws per sample (Steele, Lea, Flood 2014), draw 0 sets the
   edge threshold t in [26, 128] (p = t/256 in [0.1, 0.5]), edge e is present
   iff byte e%8 of draw 1+e/8 is below t (Sec. 7, Erdos-Renyi frames). */
uint64_t mk_sample_relation(uint64_t seed, int32_t n, uint64_t s);

/* Decode a split key into a certificate for (phi, psi) (host). */
int mk_split_cert(const mk_program *h_phi, const mk_program *h_psi, const char *phi,
                  const char *psi, uint64_t seed, uint32_t samples,
                  const uint32_t *h_samples_n, uint64_t key, mk_cert *out);

/* Kernel launches one mk_census call with this configuration issues
   (result initialisation, class-list construction, one per layer). */
int32_t mk_census_launches(const mk_census_cfg *cfg, int32_t nprog);

/* ------------------------------------------------------ calibration */
/* Logic-op issue ceiling (the roofline denominator of the census; Sec. 8
   measures the same uint32 logic ceiling): launches blocks x threads
   threads, each running independent chains of three-input logic ops for
   `iters` iterations; d_sink is a device word array of `blocks` entries. */
int mk_calibrate_lop3(uint32_t *d_sink, int32_t blocks, int32_t threads, uint32_t iters,
                      uint32_t seed, void *stream);
/* Logic ops one such launch performs. */
uint64_t mk_calibrate_ops_per_launch(int32_t blocks, int32_t threads, uint32_t iters);

/* ------------------------------------------------------ learned proposal */
/* Truth vectors and the pair-ranking MLP.  Sec. 9 ranks candidate pairs by
   small-frame semantic representations and verifies every hit exactly; here
   the representation is a truth vector and the ranking a small MLP trained
   on pairs the exact search has labelled.  The exact separation search
   (mk_separate) and mk_certify remain the only judges of a hit. */
typedef struct {
    uint64_t frame;        /* K index of the model's frame                  */
    uint32_t val;          /* valuation value (p_i at w: bit i*n+w)          */
    uint8_t n;             /* worlds, 1..6                                   */
    uint8_t world;         /* pointed world                                  */
    uint16_t reserved;
} mk_model;                /* 16 bytes                                       */

/* Truth vectors: bit j of formula p's vector (word j/32 of row p, rows of
   ngroups words) = program p is true at world models[j].world of model j.
   Models come in groups of 32 with one n per group (h_group_n[g], host);
   d_models holds 32*ngroups models. */
int mk_fingerprint(const mk_program *d_progs, int32_t nprog, const mk_model *d_models,
                   const int32_t *h_group_n, int32_t ngroups, uint32_t *d_bits, int32_t *d_status,
                   void *stream);

/* Exact k nearest neighbours of every vector in Hamming distance (self
   excluded): d_nbr[q*k + i] / d_dist[q*k + i] list, for each query q, all
   vectors with distance < t and the lowest-index ones with distance == t,
   where t is the least distance reaching k neighbours; -1 / 0xFFFF pad
   when fewer than k other vectors exist.  words: 32-bit words per vector. */
size_t mk_knn_workspace_size(int32_t nvec);
int mk_hamming_knn(const uint32_t *d_bits, int32_t nvec, int32_t words, int32_t k, int32_t *d_nbr,
                   uint16_t *d_dist, void *d_workspace, size_t ws_bytes, void *stream);

/* The MLP: x = [a xor b, a and b] for the truth vectors a, b of a pair
   (features = 64 * words per vector), h1 = relu(x W1 + b1), h2 = relu(h1 W2
   + b2), logit = h2 . w3 + b3.  Parameters are one FP32 buffer in the order
   W1[features][hidden], b1, W2[hidden][hidden], b2, w3[hidden], b3.
   Pairs are given by vector indices d_pa[i], d_pb[i]. */
size_t mk_mlp_param_count(int32_t features, int32_t hidden);
size_t mk_mlp_workspace_size(int32_t batch, int32_t hidden);
int mk_mlp_forward(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                   const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits,
                   void *d_workspace, size_t ws_bytes, void *stream);
/* Gradient of the weighted binary cross-entropy sum_i w_i * BCE(logit_i, y_i)
   (d_w may be NULL for weight 1) with respect to every parameter, in the
   parameter layout, into d_grad; the loss into *d_loss.  FP32 throughout. */
size_t mk_mlp_train_workspace_size(int32_t batch, int32_t features, int32_t hidden);
int mk_mlp_gradient(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                    const int32_t *d_pa, const int32_t *d_pb, const float *d_y, const float *d_w,
                    int32_t batch, float *d_grad, float *d_loss, void *d_workspace, size_t ws_bytes,
                    void *stream);
/* One Adam step (Kingma and Ba, 2015) on n parameters; step counts from 1. */
int mk_adam_step(float *d_params, const float *d_grad, float *d_m, float *d_v, size_t n, float lr,
                 float beta1, float beta2, float eps, int32_t step, float grad_scale, void *stream);
/* Scoring with the first layer on the tensor cores in BF16 (the 0/1
   features are exact; W1 is rounded to BF16), FP32 accumulation; hidden
   must be 256. */
size_t mk_mlp_infer_workspace_size(int32_t batch, int32_t features, int32_t hidden);
int mk_mlp_infer_bf16(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                      const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits,
                      void *d_workspace, size_t ws_bytes, void *stream);

/* The same scoring with the first layer on the 5th-generation tensor cores
   (tcgen05.mma, BF16 operands in shared memory, FP32 accumulator in tensor
   memory); features a multiple of 128, hidden 256.  A bounded wait that
   runs out sets MK_ST_TIMEOUT in *d_status (the logits are then invalid). */
int mk_mlp_infer_tc(const float *d_params, int32_t features, int32_t hidden, const uint32_t *d_vec,
                    const int32_t *d_pa, const int32_t *d_pb, int32_t batch, float *d_logits, int32_t *d_status,
                    void *d_workspace, size_t ws_bytes, void *stream);

/* The first layer alone, h1[i * 256 + h] = relu(x_i . W1[:, h] + b1[h]) with
   W1 given as BF16 W1^T (d_w1t[h * features + f], from mk_mlp_w1t_bf16):
   on tcgen05 (features % 128 == 0, 16-byte aligned d_w1t and d_h1) or on
   warp-level mma.sync (the legacy path, for comparison). */
int mk_mlp_w1t_bf16(const float *d_params, int32_t features, int32_t hidden, void *d_w1t, void *stream);
int mk_mlp_layer1_tc(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                     int32_t batch, const void *d_w1t, const float *d_b1, float *d_h1, int32_t *d_status,
                     void *stream);
int mk_mlp_layer1_mma(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                      int32_t batch, const void *d_w1t, const float *d_b1, float *d_h1, void *stream);

/* The production first layer: warp-specialised (4 producer warps, 1 MMA
   warp), 256 pairs per CTA in two M=128 accumulators (all 512 TMEM
   columns), each W1 block fetched as one bulk copy from a pre-arranged
   image (mk_mlp_w1_tiles: features/64 tiles of 32 KB, the swizzled K-major
   layout the MMA reads; mk_mlp_w1_tiles_bytes gives its size). */
size_t mk_mlp_w1_tiles_bytes(int32_t features);
int mk_mlp_w1_tiles(const float *d_params, int32_t features, int32_t hidden, void *d_tiles, void *stream);
int mk_mlp_layer1_tc_ws(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                        int32_t batch, const void *d_w1_tiles, const float *d_b1, float *d_h1, int32_t *d_status,
                        void *stream);

/* The same layer with the iteration limit of its pipeline waits given by the
   caller (wait_spins >= 1 tests of an mbarrier, each followed by a ~32 ns
   sleep; mk_mlp_layer1_tc_ws uses 2^24, about two seconds).  A limit that
   runs out is the failure the bounded waits guard against (a copy or an MMA
   that never completes): the CTA's roles agree to abort, the bulk copies
   already issued are waited for on their own barriers, one more
   tcgen05.commit tracks every MMA already issued and is waited for, the
   tensor memory is freed, MK_ST_TIMEOUT is OR-ed into *d_status and h1 is
   left undefined.  The context stays usable.  A small limit makes the waits
   run out on purpose, which is how the timeout path is tested.
   MK_E_ARG for wait_spins == 0, otherwise as mk_mlp_layer1_tc_ws. */
int mk_mlp_layer1_tc_ws_bounded(const uint32_t *d_vec, int32_t features, const int32_t *d_pa, const int32_t *d_pb,
                                int32_t batch, const void *d_w1_tiles, const float *d_b1, float *d_h1,
                                int32_t *d_status, uint32_t wait_spins, void *stream);

/* ------------------------------------------- large frames (Sec. 7) */
/* Separation beyond the exhaustive sizes runs over explicit relations on up
   to 16 worlds: the 39 stress templates (path, reverse-path, reflexive-path,
   fork, cycle, star, sparse and dense frames) used to challenge pairs that
   agree on every small frame, and the six adversarial relation generators
   of Table 2.  The paper names these families without fixing their
   construction; mk_template and mk_stress_relation define the ones used
   here (their readings are listed with the design notes).  A relation is a
   list of successor masks: bit v of succ[w] is set iff R(w, v). */
#define MK_MAX_WORLDS_STRESS 16
#define MK_NUM_TEMPLATES 39
enum {
    MK_GEN_ER = 0,        /* Erdos-Renyi, per-relation p in [0.1, 0.5]      */
    MK_GEN_FLIP = 1,      /* 1..4 edge flips of a random template           */
    MK_GEN_SCC = 2,       /* two strongly connected blocks, one bridge      */
    MK_GEN_DEADEND = 3,   /* Erdos-Renyi with 1..3 worlds made dead ends    */
    MK_GEN_BACKEDGE = 4,  /* the path plus 1..4 backward edges              */
    MK_GEN_PERMSCC = 5,   /* SCC bottleneck with the worlds relabelled      */
    MK_NUM_GENERATORS = 6
};

/* Template id (0..38) on n worlds (1..16), host: succ[0..n). */
int mk_template(int32_t id, int32_t n, uint32_t *succ);

/* Relation s of generator gen on n worlds (host): every relation is a
   function of (gen, seed, n, s) alone, drawn from SplitMix64 streams; for
   MK_GEN_ER and n <= 8 it is mk_sample_relation(seed, n, s).  n: 1..16 for
   MK_GEN_ER, 2..16 otherwise. */
int mk_stress_relation(int32_t gen, uint64_t seed, int32_t n, uint64_t s, uint32_t *succ);

/* Relation words: relations are evaluated 32 at a time, bit-sliced.  Block
   b of a relation list holds relations 32b .. 32b+31; its word (w, v) is
   d_words[(b * n + w) * n + v], whose bit l is R(w, v) of relation 32b + l
   (zero past the end of the list).  mk_relation_words gives the number of
   uint32 words for `count` relations. */
uint64_t mk_relation_words(int32_t n, uint64_t count);

/* Generate relations first .. first+count-1 of generator gen on the device:
   their words into d_words (may be NULL) and their successor masks into
   d_succ[i * 16 + w] (may be NULL; rows w >= n are zero). */
int mk_generate_relations(int32_t gen, uint64_t seed, int32_t n, uint64_t first, uint64_t count,
                          uint32_t *d_words, uint32_t *d_succ, void *stream);

/* Pack a caller's relation list (d_succ[i * 16 + w], i < count) into words. */
int mk_pack_relations(const uint32_t *d_succ, int32_t n, uint64_t count, uint32_t *d_words,
                      void *stream);

typedef struct {
    int32_t n;             /* worlds of every relation, 1..16                */
    int32_t count_splits;  /* 1: also count, per pair, the relations that   */
                           /* split it (d_nsplit); 0: first split only, and  */
                           /* a pair whose key already lies below every key  */
                           /* a CTA could produce is skipped by that CTA     */
    uint64_t count;        /* relations in d_words                           */
    uint64_t index_base;   /* relation index of the list's first relation    */
    mk_tune tune;          /* tile: pairs per CTA, 1..64 (0 = 16)            */
} mk_stress_cfg;

/* Separation over a relation list (Def. 2, Prop. 4 on explicit frames): for
   each pair i, the least (relation, valuation, world) at which phi_i and
   psi_i differ, relations in list order, valuations exhaustive
   (x = 0 .. 2^(k n)-1, which requires k*n <= 16; a pair beyond that sets
   MK_ST_LIMIT and is skipped), merged into d_key[i] by atomic minimum as
       (index_base + position) << 20 | x << 4 | w
   (d_key must hold UINT64_MAX or an earlier call's key; positions < 2^44).
   With count_splits, d_nsplit[i] (cleared by the caller) is increased by the
   number of relations on which the pair differs for some valuation. */
int mk_stress_separate(const mk_program *d_phi, const mk_program *d_psi, int32_t npairs,
                       const uint32_t *d_words, const mk_stress_cfg *cfg, uint64_t *d_key,
                       uint32_t *d_nsplit, int32_t *d_status, void *stream);

/* --------------------------------------- frame correspondents (Sec. 10) */
/* Recovering a first-order frame condition for a formula (Sec. 10, Table
   9): over every frame of n <= N worlds, the frames that validate the
   formula (true at every world under every valuation) are compared with
   the frames that satisfy a condition of a fixed library; a condition
   whose extension is equal on all of them is the recovered correspondent.
   Bitmaps are over the K index: bit f%32 of word f/32 is frame f. */
#define MK_MAX_WORLDS_VALIDITY 5
enum {
    MK_COND_ALL = 0,          /* every frame                                */
    MK_COND_NONE = 1,         /* no frame                                   */
    MK_COND_REFLEXIVE = 2,    /* wRw                                        */
    MK_COND_IRREFLEXIVE = 3,  /* not wRw                                    */
    MK_COND_SERIAL = 4,       /* exists v: wRv                              */
    MK_COND_TRANSITIVE = 5,   /* wRv, vRu => wRu                            */
    MK_COND_SYMMETRIC = 6,    /* wRv => vRw                                 */
    MK_COND_EUCLIDEAN = 7,    /* wRv, wRu => vRu                            */
    MK_COND_PARTFUNC = 8,     /* wRv, wRu => v = u                          */
    MK_COND_FUNCTIONAL = 9,   /* exactly one successor                      */
    MK_COND_DENSE = 10,       /* wRv => exists u: wRu, uRv                  */
    MK_COND_DIRECTED = 11,    /* wRv, wRu => exists x: vRx, uRx             */
    MK_COND_ANTISYM = 12,     /* wRv, vRw => w = v                          */
    MK_COND_ASYM = 13,        /* wRv => not vRw                             */
    MK_COND_CONNECTED = 14,   /* wRv, wRu => vRu or v = u or uRv            */
    MK_COND_SHIFTREFL = 15,   /* wRv => vRv                                 */
    MK_COND_EMPTY = 16,       /* no edge                                    */
    MK_COND_COREFLEXIVE = 17, /* wRv => w = v                               */
    MK_NUM_CONDITIONS = 18
};

/* Words of one n-world bitmap: ceil(2^(n*n) / 32); 0 if n is out of range. */
uint64_t mk_frame_words(int32_t n);

/* d_bits[p * ld_words + word]: validity bitmap of program p over the
   n-world frames (1 <= n <= 5), all valuations exhaustive (k*n <= 24, else
   MK_ST_LIMIT and the row is left unwritten); bits past 2^(n*n) are 0.
   max_depth: largest program depth (0 = MK_MAX_STACK), as in the census. */
int mk_frame_validity(const mk_program *d_progs, int32_t nprog, int32_t n, int32_t max_depth,
                      uint32_t *d_bits, uint64_t ld_words, int32_t *d_status, void *stream);

/* d_bits[c * ld_words + word]: extension of library condition c over the
   n-world frames, for every c < MK_NUM_CONDITIONS. */
int mk_frame_conditions(int32_t n, uint32_t *d_bits, uint64_t ld_words, void *stream);

/* d_out[i * nconj + j] = number of frames (set bits among the first
   `words` words) where row i of d_a differs from the conjunction of rows
   d_conj[2j] and d_conj[2j+1] of d_b (equal indices: one condition);
   UINT32_MAX if an index is outside 0..nb-1. */
int mk_bitmap_mismatch(const uint32_t *d_a, int32_t na, uint64_t lda, const uint32_t *d_b, int32_t nb,
                       uint64_t ldb, const int32_t *d_conj, int32_t nconj, uint64_t words, uint32_t *d_out,
                       void *stream);

/* ------------------------------------------ failure-density atlas (Sec. 9) */
/* D_ij = the fraction of (valuation, world) pairs at which formula i is
   false on frame j, over all 2^(n*n) frames (the paper's atlas uses the 512
   three-world frames); its seriation (centre the columns, order frames by
   the first principal axis and formulas by their coordinate on it), the
   adjacent variation A(pi) = sum_i sum_j |D_i,pi(j+1) - D_i,pi(j)| /
   (B (F-1)), and the 2-D density view (binned points). */

/* d_counts[p * ld + f]: the numerator of D for program p on frame f
   (1 <= n <= 4); the denominator is 2^(k n) * n with k = the program's
   nvars (valuations exhaustive, k*n <= 16 else MK_ST_LIMIT). */
int mk_atlas_counts(const mk_program *d_progs, int32_t nprog, int32_t n, uint32_t *d_counts, uint64_t ld,
                    int32_t *d_status, void *stream);

#define MK_MAX_ATLAS_AXIS 4096   /* frames F for the Gram matrix (n <= 3: 512) */

/* Column means of D (d_mean[F]) and the centred Gram matrix
   d_gram[a * F + b] = sum_i (D_ia - m_a)(D_ib - m_b), FP64; d_denom[B]. */
int mk_atlas_gram(const uint32_t *d_counts, const uint64_t *d_denom, int32_t B, int32_t F, uint64_t ld,
                  double *d_mean, double *d_gram, void *stream);

/* Leading eigenvector d_v[F] (and its Rayleigh quotient) of the symmetric
   matrix d_gram, orthogonal to the nprev vectors d_prev[nprev * F], by
   at most `iters` power-iteration steps from a fixed start (fewer once a
   step moves it by less than 1e-14); its largest-magnitude component is
   positive.  One CTA; F <= MK_MAX_ATLAS_AXIS.  The workspace is unused
   (kept for the calling convention; its size may be 0). */
size_t mk_power_workspace_size(int32_t F);
int mk_power_iteration(const double *d_gram, int32_t F, const double *d_prev, int32_t nprev, int32_t iters,
                       double *d_v, double *d_lambda, void *d_workspace, size_t ws_bytes, void *stream);

/* Formula coordinates d_u[i] = sum_j (D_ij - m_j) v_j. */
int mk_atlas_project(const uint32_t *d_counts, const uint64_t *d_denom, int32_t B, int32_t F, uint64_t ld,
                     const double *d_mean, const double *d_v, double *d_u, void *stream);

/* d_order: the indices 0..n-1 sorted by (d_keys[i], i) ascending. */
size_t mk_sort_workspace_size(int32_t n);
int mk_sort_keys(const double *d_keys, int32_t n, int32_t *d_order, void *d_workspace, size_t ws_bytes,
                 void *stream);

/* d_rowsum[i] = sum_j |count_i,perm(j+1) - count_i,perm(j)| (exact; A(pi) =
   sum_i rowsum_i / denom_i / (B (F-1))).  A perm entry outside 0..F-1 sets
   MK_ST_INDEX and its term is skipped. */
int mk_adjacent_variation(const uint32_t *d_counts, int32_t B, int32_t F, uint64_t ld, const int32_t *d_perm,
                          uint64_t *d_rowsum, int32_t *d_status, void *stream);

/* d_hist[G * G] (cleared first): point i falls in column
   floor((x_i - lo) / (hi - lo) * G) and row floor((y_i - lo) / (hi - lo) * G),
   in FP64, clamped to 0..G-1 (NaN to 0). */
int mk_histogram2d(const double *d_x, const double *d_y, int64_t npts, double lo, double hi, int32_t G,
                   uint32_t *d_hist, void *stream);

/* d_stats[4] = occupied cells, largest cell, points in cells holding more
   than one point, cells within Chebyshev distance `radius` of an occupied
   cell (the pixels square marks of that radius would cover). */
int mk_histogram_stats(const uint32_t *d_hist, int32_t G, int32_t radius, uint64_t *d_stats, void *stream);

/* ------------------------------------------------------------- misc */
const char *mk_strerror(int code);
int mk_status_error(int32_t status);   /* MK_OK or the MK_E_* for status bits */
int mk_version(void);                  /* ABI version                         */

#ifdef __cplusplus
}
#endif
#endif /* MK_H */
