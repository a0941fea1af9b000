// ohm_internal.h -- device-side tables and kernel launchers shared by the host orchestration
// (ohm_host.cpp) and the kernels (ohm_kernels.cu).  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace ohm {

constexpr int BS = 8;      // cells per block edge
constexpr int B3 = 512;    // cells per block
constexpr int TS = 10;     // staged tile edge (block + 1-cell halo)
constexpr int T3 = 1000;   // staged tile cells

// Device tables of one blocked grid (an AMR level or a base multigrid grid).  Block indices
// inside a grid are local (0..nblk-1); field pointers handed to kernels are offset to the
// grid's first block.
struct GridDev {
    int nblk = 0;
    int level_shift = 0;            // AMR level (0 for base multigrid grids)
    double h = 0;                   // cell width
    int dims[3] = {0, 0, 0};        // cells per axis of the whole grid domain
    const int *nbr = nullptr;       // [nblk][27] same-grid neighbour or -1 (absent)
    const uint8_t *covered = nullptr;  // [nblk] 1 if refined by the next AMR level
    const int *gslot = nullptr;     // [nblk] ghost slot or -1 (AMR levels >= 1)
    const int *parent = nullptr;    // [nblk] index in the coarser grid (or -1)
    const uint8_t *octant = nullptr;// [nblk] (bi&1) | (bj&1)<<1 | (bk&1)<<2
    const int *child = nullptr;     // [nblk][8] index in the finer AMR level or -1
    const int *origin = nullptr;    // [nblk][3] block coordinates (bi, bj, bk)
    const int *freg = nullptr;      // [nblk][6] flux-register slot for faces with no neighbour
    const int *rsrc = nullptr;      // [nblk][6] index into the reflux source table or -1
    const int *slot_block = nullptr;// [nslot] block owning each ghost slot
    int nslot = 0;
    int slot0 = 0;                  // first ghost slot of this grid in the global slot array
    int inst_nblk = 0;              // batched hierarchies: blocks per instance (instance of block b
                                    // = b / inst_nblk); 0 = one instance
    const uint8_t *imask = nullptr; // batched inner iterations: thread blocks of instances whose
                                    // flag is 0 return at once (their results are not used)
    double omega = 1.0;             // relaxation factor of the red-black sweeps (1 = Gauss-Seidel)
};

// Lexicographic coarse grids below the last blocked grid (solved in one thread block).
constexpr int MAX_SMALL = 12;
template <typename T>
struct SmallDev {
    int n = 0;                      // number of small grids
    int ninst = 1;                  // instances; the arrays of grid s hold them one after another
                                    // (instance q at q * ncomp * cells(s)), one thread block each
    const uint8_t *imask = nullptr; // k_bottom skips instances whose flag is 0
    double omega = 1.0;             // relaxation factor folded into inv (1 = Gauss-Seidel)
    int dims[MAX_SMALL][3];
    double h[MAX_SMALL];
    T *e[MAX_SMALL], *r[MAX_SMALL], *t[MAX_SMALL], *eta[MAX_SMALL], *inv[MAX_SMALL];
};

// ------------------------------------------------------------------ kernel launchers
// Every launcher enqueues on `s` and returns cudaGetLastError().
// Composite operator on AMR level g (float64): out = a X + c divF(X) + d Y on leaf blocks,
// reading ghosts from Gx (level ghost slots) and eta ghosts from Geta; writes face fluxes to
// registers for faces without a same-level neighbour and reads refluxed fluxes from the
// finer level for faces next to covered blocks; optional per-block norm partials.
// Computed in TC; out (and out2 when not null) receive the result as TO.
// With outS (first residual of a step, Eqs. 14 and 20 from one flux divergence of X = b):
// outS = a X + c divF(X) (the source S) and out = out2 = c2 divF(X) = S - L X for c2 = -dt;
// the norm partials are then those of out against S.
template <typename TC, typename TO>
cudaError_t launch_composite(const GridDev &g, const TC *X, const TC *Y, const TC *eta, const TC *Gx,
                             const TC *Geta, double a, double c, double d, TO *out, TO *out2,
                             double *reg, const int *rsrc_tab, double *partials, double vol,
                             cudaStream_t s, double *outS = nullptr, double c2 = 0.0);

// Float-float number: the unevaluated sum hi + lo of two float32 values (about 48 significant
// bits).  The mixed-precision path evaluates its outer residual in this arithmetic on the
// float32 pipe and keeps the source S of a step in this form (8 bytes per value, like float64).
struct alignas(8) dfloat {
    float hi, lo;
#ifdef __CUDACC__
    __host__ __device__
#endif
    constexpr explicit dfloat(float h = 0.f, float l = 0.f) : hi(h), lo(l) {}
};

// launch_composite for the outer residual of the mixed path: X, eta and the ghosts are float64
// fields, split into float-float values when staged; Y and outS are the source in float-float
// form; out / out2 are float32 (the inner solve's right-hand side).  Float-float arithmetic
// keeps the error of R = S - L X near 2^-48 (1 + lambda dt |divF| / |X|) |X|, which bounds the
// relative residual the mixed path can certify; norm partials are accumulated in float32.
cudaError_t launch_composite_df(const GridDev &g, const double *X, const dfloat *Y, const double *eta,
                                const double *Gx, const double *Geta, double a, double c, double d, float *out,
                                float *out2, double *reg, const int *rsrc_tab, double *partials, double vol,
                                cudaStream_t s, dfloat *outS, double c2);
// the same float-float evaluation with Y a float64 field (split into float-float values as it
// is read); no source output
cudaError_t launch_composite_df(const GridDev &g, const double *X, const double *Y, const double *eta,
                                const double *Gx, const double *Geta, double a, double c, double d, float *out,
                                float *out2, double *reg, const int *rsrc_tab, double *partials, double vol,
                                cudaStream_t s);

template <typename T>
cudaError_t launch_smooth(const GridDev &g, const T *e_in, T *e_out, const T *r, const T *eta,
                          const T *inv, const T *Ge, const T *Geta, double lamdt, int colour,
                          cudaStream_t s);

// One full red + black sweep in one launch (grids without coarse-fine ghosts), inverse
// diagonal formed on the fly; e_in != e_out.
template <typename T>
cudaError_t launch_smooth_rb(const GridDev &g, const T *e_in, T *e_out, const T *r, const T *eta, double lamdt,
                             cudaStream_t s);

// The same sweep for pairs of x-adjacent blocks (2q, 2q+1): grids with an even block count whose
// pairs are x-neighbours and whose blocks all have their 26 neighbours.  e_in = nullptr: the
// sweep starts from e = 0 (nothing is read for e).
cudaError_t launch_smooth_rb2(const GridDev &g, const float *e_in, float *e_out, const float *r, const float *eta,
                              double lamdt, cudaStream_t s);
// float32 operator or residual on block pairs of a brick grid (every block pair x-adjacent, all
// neighbours present): apply: out = X + kc divF(X); else out = (Y - X) + kc divF(X) (out may be
// null) with, when coarse is not null, its octet means written into the coarser grid (children
// in Morton octets: block b's parent b / 8, octant b % 8)
cudaError_t launch_pair_op(const GridDev &g, const float *X, const float *Y, const float *eta, double kc, bool apply,
                           float *out, float *coarse, cudaStream_t s);

// t = r - (e + lamdt divF(e)); restricted (mean of 8) into the coarser grid: blocked
// (coarse != nullptr, by parent/octant) or lexicographic (lex != nullptr, dims ldims).
template <typename T>
cudaError_t launch_resid_restrict(const GridDev &g, const T *e, const T *r, const T *eta,
                                  const T *Ge, const T *Geta, double lamdt, T *t_out,
                                  T *coarse, T *lex, const int *ldims, cudaStream_t s);

template <typename T>
cudaError_t launch_prolong_add(const GridDev &g, const GridDev *gc, const T *coarse,
                               const T *lex, const int *ldims, T *fine, int *err, cudaStream_t s);

// the same for a coarse grid gc whose blocks' children are the fine blocks 8c .. 8c+7 in
// octant order (one thread block per coarse block)
template <typename T>
cudaError_t launch_prolong_add8(const GridDev &gc, const T *coarse, T *fine, cudaStream_t s);

// plain restriction of ncomp components (eta chain): blocked fine -> blocked or lex coarse
template <typename T>
cudaError_t launch_restrict(const GridDev &g, const T *fine, int ncomp, T *coarse, T *lex,
                            const int *ldims, cudaStream_t s);

template <typename TS, typename TD>
cudaError_t launch_ghost_fill(const GridDev &g, const GridDev &gc, const TS *coarse, int ncomp,
                              TD *ghost, int *err, cudaStream_t s);

template <typename T>
cudaError_t launch_sync_down(const GridDev &gc, T *Bc, const T *Bf, cudaStream_t s);

// x += y / B += e on leaf blocks; with imask, only on blocks of instances whose flag is set
template <typename T>
cudaError_t launch_axpy_leaf(const GridDev &g, T *x, const T *y, const uint8_t *imask, cudaStream_t s);

template <typename T>
cudaError_t launch_update(const GridDev &g, double *B, const T *e, const uint8_t *imask, cudaStream_t s);

// Per-instance norms of a batched hierarchy: instance q owns blocks [off[l] + q n[l],
// off[l] + (q+1) n[l]) of every level l; out[q] = {sum R^2 dV, sum S^2 dV, max |R|, 0},
// each folded in a fixed order that does not depend on the other instances.
constexpr int MAX_LEVELS_DEV = 8;
struct InstRanges {
    int nlev = 0;
    int off[MAX_LEVELS_DEV];
    int n[MAX_LEVELS_DEV];
};
cudaError_t launch_norm_inst(const double *partials, const InstRanges &R, int ninst, double *out, cudaStream_t s);

// dst[b][512] = src[b][512] * scale[b] (per-block scale of a block field)
cudaError_t launch_scale_blocks(const double *src, double *dst, const double *scale, int nblk, cudaStream_t s);

template <typename T>
cudaError_t launch_invdiag(const GridDev &g, const T *eta, const T *Geta, double lamdt, T *inv,
                           cudaStream_t s);

// scratch: NORM_SCRATCH_BYTES, zero-filled once before first use (it resets itself)
constexpr size_t NORM_SCRATCH_BYTES = 128 * 3 * sizeof(double) + 16;
// host_out (optional): pinned host memory mapped into the device that also receives the three
// sums and, as an int at host_out + 4, the word *err (the caller reads them after synchronising,
// without a copy)
cudaError_t launch_norm_reduce(const double *partials, int nblocks, double *scratch, double *out, cudaStream_t s,
                               double *host_out = nullptr, const int *err = nullptr);

template <typename T>
cudaError_t launch_bottom(const SmallDev<T> &sm, double lamdt, int nu_pre, int nu_post,
                          int n_coarse, cudaStream_t s);
// whether launch_bottom runs these float32 grids in the shared-memory solver (every extent a
// power of two, the grids within its shared memory), which forms the diagonal from eta and does
// not read the grids' inverse diagonals
bool bottom_in_shared(const SmallDev<float> &sm);

// Grid-wide steps on lexicographic grid s of every instance (grids too large for the one-block
// coarsest solver): nsweep red-black sweeps (e -> t -> e), residual into t and its restriction
// into r of grid s + 1 (e of grid s + 1 zeroed), prolongation e_s += P e_{s+1}.
template <typename T>
cudaError_t launch_lex_sweeps(const SmallDev<T> &sm, int s, double lamdt, int nsweep, cudaStream_t st);
template <typename T>
cudaError_t launch_lex_resid_restrict(const SmallDev<T> &sm, int s, double lamdt, cudaStream_t st);
template <typename T>
cudaError_t launch_lex_prolong(const SmallDev<T> &sm, int s, cudaStream_t st);

// lexicographic restriction between small grids and small-grid inverse diagonals
template <typename T>
cudaError_t launch_small_setup(const SmallDev<T> &sm, double lamdt, bool eta_chain, cudaStream_t s);

template <typename TS, typename TD>
cudaError_t launch_convert(const TS *src, TD *dst, size_t n, cudaStream_t s);

// *flag = 1 if the n float64 values of a and b differ in any bit (flag is not cleared here)
cudaError_t launch_differs(const double *a, const double *b, size_t n, int *flag, cudaStream_t s);

// Krylov vector operations (float32 fields [nblk][3][512]); at most KMAX vectors at once.
constexpr int KMAX = 12;
struct VecSet {
    const float *v[KMAX];
    float c[KMAX];
    int k = 0;
};
// out[0..k-1] = <w, v_i>, out[k] = <w, w>, volume weighted per block by wb (0 = excluded);
// part: scratch of nblk * (k + 1) doubles.  gate (device, may be null): when it holds 0 the
// launches return at once and out is left as it was.
cudaError_t launch_mdot(const float *w, const VecSet &V, const double *wb, int nblk, double *part, double *out,
                        cudaStream_t s, const int *gate = nullptr, double *host_out = nullptr);
// w = X + kc divF(X) on the block pairs of a single-level brick grid (launch_pair_op's operator)
// with out[0..k-1] = <w, v_i> and out[k] = <w, w>, every cell weighted by wt; part: scratch of
// (nblk / 2) * (k + 1) doubles; host_out as for launch_mdot
cudaError_t launch_pair_apply_dots(const GridDev &g, const float *X, const float *eta, double kc, float *w,
                                   const VecSet &V, double wt, double *part, double *out, double *host_out,
                                   cudaStream_t s);

// dst = (src - sum c_i v_i) * scale; src null stands for 0
cudaError_t launch_maxpy(float *dst, const float *src, const VecSet &V, float scale, size_t n, cudaStream_t s);

// The same Krylov vector operations on float64 vectors (the float64 FGMRES of OHM_FP64)
struct VecSetD {
    const double *v[KMAX];
    double c[KMAX];
    int k = 0;
};
cudaError_t launch_mdot(const double *w, const VecSetD &V, const double *wb, int nblk, double *part, double *out,
                        cudaStream_t s, double *host_out = nullptr);
cudaError_t launch_maxpy(double *dst, const double *src, const VecSetD &V, double scale, size_t n, cudaStream_t s);

cudaError_t launch_zero_covered(const GridDev &g, double *x, cudaStream_t s);

// Per-instance FGMRES(m) scalars of a batched hierarchy, kept on the device so that a whole
// restart cycle is a fixed sequence of launches (capturable in a CUDA graph): Hessenberg
// columns, Givens rotations, residual estimates and the stopping decisions, one thread per
// instance.  dots are the products of the last multi-dot ([K][KMAX+1]); coef receives the
// coefficients of the next multi-axpy ([K][KMAX+1], scale in the last entry); imask is the
// compute mask of the V-cycle and operator kernels.
struct FgState {
    double *Hm = nullptr;                      // [K][KMAX+1][KMAX]
    double *cs = nullptr, *sn = nullptr;       // [K][KMAX]
    double *g = nullptr;                       // [K][KMAX+1]
    double *beta0 = nullptr, *beta = nullptr, *brest = nullptr, *target = nullptr, *hn = nullptr;  // [K]
    int *cycles = nullptr, *jend = nullptr;    // [K]
    uint8_t *live = nullptr, *arn = nullptr, *act = nullptr, *need2 = nullptr, *run = nullptr;  // [K]
    uint8_t *imask = nullptr;                  // [K]
    const double *dots = nullptr;
    float *coef = nullptr;
    int *any_need2 = nullptr;                  // 1 when some instance needs the norm pass of the step
    int K = 0, m = 0, max_outer = 0;
};
enum FgOp { FG_START, FG_CYCLE, FG_ACT, FG_ORTHO, FG_RENORM, FG_GIVENS, FG_SOLVE, FG_RESTART_MASK, FG_RESTART };
cudaError_t launch_fg(const FgState &f, FgOp op, int j, cudaStream_t s);

// Batched hierarchies: per-instance products out[q][0..k] (layout [ninst][KMAX+1]; part:
// nblk * (k+1) doubles of block partials), and dst = (src - sum_i coef[q][i] v_i) * coef[q][KMAX]
// with q = binst[block] (coef: [ninst][KMAX+1] floats on the device).
// gate as for launch_mdot.
cudaError_t launch_mdot_inst(const float *w, const VecSet &V, const double *wb, int nblk, const InstRanges &R, int ninst,
                             double *part, double *out, cudaStream_t s, const int *gate = nullptr);
cudaError_t launch_maxpy_inst(float *dst, const float *src, const VecSet &V, const float *coef, const int *binst,
                              size_t n, cudaStream_t s, const int *gate = nullptr);

}  // namespace ohm
