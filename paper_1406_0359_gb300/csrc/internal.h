// Internal data layout and kernel launchers of the GB300 SARA-SDMM path.
//
// HBM layout of one operator (T = float or double, C = complex<T>):
//   pos    [M]        visibility positions in uv-tile order (Pos<T>)
//   perm   [M]        sorted slot -> caller's visibility index
//   items  [n_items]  work items: (tile, first slot, end slot), <= chunk slots each
//   gridA  [n][K/2]   half-spectrum rows: the row FFTs of image row pairs
//                     x_a + i x_b split into the half spectra of rows a and b
//                     (entry 0 = X(0) + i X(K/2)), after the forward row pass
//                     or before the inverse one
//   gridP  [KP][KP]   forward oversampled grid with a J-wide periodic halo,
//                     read in (TB+J)^2 patches by TMA for degridding
//   gridQ  [KP][KP]   gridding accumulator with the same halo (folded on read)
// with K = 2n the oversampled grid side and KP = K + J its padded side.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "common.cuh"

namespace purify {

constexpr int kJ = 8;           // Kaiser-Bessel support (taps per axis)
constexpr int kDegF = 10;       // kernel polynomial degree, FP32 path
constexpr int kDegD = 16;       // kernel polynomial degree, FP64 path
constexpr int kMaxDb = 8;       // Db1..Db8
constexpr int kMaxTaps = 16;    // Db8 length

template <typename T> struct KbDeg;
template <> struct KbDeg<float> { static constexpr int value = kDegF; };
template <> struct KbDeg<double> { static constexpr int value = kDegD; };

// Kernel polynomial coefficients, tap-major: c[a][d] for x = 2f - 1.
template <typename T> struct KbPoly { T c[kJ][KbDeg<T>::value + 1]; };

// Encoded grid position of one visibility inside its uv tile.
// FP32: 8 integer bits of cell + 24 fraction bits per axis (6e-8 cell resolution).
// FP64: the tile-local coordinate itself.
template <typename T> struct Pos;
template <> struct Pos<float> { uint32_t u, v; };
template <> struct Pos<double> { double u, v; };

struct WorkItem { int tile, begin, end, pad; };  // pad: visibility block of the item

struct Geometry {
  int n, K, KP, pad_lo, TB, ntile1d;
  int64_t M;
};

// Daubechies analysis filters h (low) and g (high), zero-padded to 16 taps.
template <typename T> struct DbFilters { T h[kMaxDb][kMaxTaps]; T g[kMaxDb][kMaxTaps]; };

// Row-pass epilogues (inverse row FFT -> image): val = Re(.) * s[i1] s[i2].
enum RowEpMode : int {
  EP_STORE = 0,     // out = val
  EP_CG_AP = 1,     // out = nu2 val + 2 p (= A p);  partials <p,Ap>, <r,Ap>, <Ap,Ap>, <r,p>, <r,r>
  EP_CG_R0 = 2,     // out = b - (nu2 val + 2 p); out2 = out; partial += out^2
  EP_POWER = 3,     // out = val;                      partial += val^2
  EP_XS_ADD = 4,    // out = b + nu val   (b may alias out)
  EP_QX = 5         // out = nu2 val + 2 p
};
template <typename T> struct RowEp {
  int mode;
  T* out;
  T* out2;
  const T* p;
  const T* b;
  const T* r;        // EP_CG_AP: the CG residual
  double nu, nu2;
  double* partials;  // per-CTA partial sums; the k-th sum at partials + k * pstride
  size_t pstride;
  // Device scalars (solver slots) finalised by the last block when ticket is
  // set: EP_CG_R0 sets S_RR; EP_CG_AP sets S_PAP, S_ALPHA = <r,p> / <p,Ap>,
  // S_BETA and the next <r,r> (from the five sums, see fft.cu).
  double* scalars;
  unsigned int* ticket;
  int* err;          // device error flag (timed-out operand staging)
};

// Forward row-pass prologues (image -> row FFT input).
enum RowProMode : int {
  PRO_PLAIN = 0,    // src = x
  PRO_CG_STEP = 1,  // x += alpha p, r -= alpha Ap, p = r + beta p (scalars S_ALPHA, S_BETA); src = p
  PRO_SCALE = 2,    // src = x * scalars[scale_idx]   (power iteration normalisation)
  PRO_CG_START = 3  // r = x - ap (b - A x_hat, A x_hat kept from the previous iteration), p = r; src = p
};
template <typename T> struct RowPro {
  int mode;
  const T* x;
  T* p;
  T* r;
  T* xu;        // PRO_CG_STEP: the CG iterate
  const T* ap;  // PRO_CG_STEP: A p of the previous step
  const double* scalars;
  int idx;
};

// Degridding epilogues (per visibility slot i, value acc = (G F Z S x)_i).
enum DegridMode : int {
  DG_STORE_PERM = 0,  // y[perm[i]] = acc
  DG_STORE_SORTED = 1,// y[i] = acc
  DG_BALL = 2         // v = nu acc + z[i]; z[i] = v; partials: |v - nu y_i|^2, |acc - y_i|^2
};
template <typename C> struct DegridEp {
  int mode;
  C* y;
  C* z;
  const C* ys;
  double nu;
  double* part0;
  double* part1;
};

// Gridding prologues (value u scattered for slot i).
enum GridMode : int {
  GP_PERM = 0,        // u = y[perm[i]]
  GP_SORTED = 1,      // u = y[i]
  GP_BALL = 2         // v = z[i], c = nu ys[i]; r = c + (v - c) * scale; z[i] = v - r; u = 2r - v
};
template <typename C> struct GridPro {
  int mode;
  const C* y;
  C* z;
  const C* ys;
  double nu;
  const double* scalars;
  int scale_idx;
  const double* block_scale;  // per visibility block (R > 1), else null
};

// Arguments of the real-form FFT passes (one operator; a batch passes a
// device table of them, one per instance).
template <typename T> struct RowFwdArgs {
  Geometry g;
  RowPro<T> pro;
  const T* deapod;
  typename cplx_t<T>::type* B;
  const typename cplx_t<T>::type* tw;
  int nseq;
};
template <typename T> struct ColConvArgs {
  Geometry g;
  typename cplx_t<T>::type* B;
  const T* khat;
  const T* knyq;
  const typename cplx_t<T>::type* tw;
  int cw;
};
template <typename T> struct RowInvArgs {
  Geometry g;
  const typename cplx_t<T>::type* B;
  const T* deapod;
  RowEp<T> ep;
  const typename cplx_t<T>::type* tw;
  int nseq;
  int nblocks;  // CTAs of the instance (its epilogue partials, its ticket)
};
template <typename T> struct ColFwdArgs {
  Geometry g;
  const typename cplx_t<T>::type* B;
  typename cplx_t<T>::type* Pg;
  const typename cplx_t<T>::type* tw;
  int cw;
};
template <typename T> struct ColInvArgs {
  Geometry g;
  const typename cplx_t<T>::type* Q;
  typename cplx_t<T>::type* B;
  const typename cplx_t<T>::type* tw;
  int cw;
};

// Arguments of the warp-per-item degridding / gridding (one operator; a batch
// passes a device table; the kernel polynomial is shared).  map: the TMA
// descriptor of the padded forward grid in global memory (batch only).
template <typename T> struct DegridArgs {
  Geometry g;
  const CUtensorMap* map;
  const WorkItem* items;
  int n_items;
  const Pos<T>* pos;
  const int* perm;
  DegridEp<typename cplx_t<T>::type> dep;
  int* err;
};
template <typename T> struct GridArgs {
  Geometry g;
  const WorkItem* items;
  int n_items;
  const Pos<T>* pos;
  const int* perm;
  GridPro<typename cplx_t<T>::type> gpro;
  typename cplx_t<T>::type* Q;
};

// Record the detail returned by purify_last_error() on this thread.
void set_last_error(const char* msg);

// First-phase budget of the bounded mbarrier waits in each compiled module
// that waits (current device).
cudaError_t set_wait_spins_fft(uint32_t spins);
cudaError_t set_wait_spins_nufft(uint32_t spins);
cudaError_t set_wait_spins_solver(uint32_t spins);
// Bounded-wait self-test: one CTA arms an mbarrier for 16 bytes and either
// delivers them by a bulk copy (deliver != 0) or sends nothing; *timed_out
// receives whether the wait gave up.  Blocks on `s`.
cudaError_t wait_selftest(int deliver, cudaStream_t s, int* timed_out);

// ----------------------------------------------------------------- launchers
// Raise the dynamic shared-memory limit of every kernel (once per operator,
// outside any stream capture).
template <typename T> cudaError_t configure_fft();
template <typename T> cudaError_t configure_nufft();
template <typename T> cudaError_t configure_sara();

// CTAs of one inverse row pass (the partial sums its epilogue writes).
int row_inv_blocks(const Geometry& g);
// Row pairs per CTA of the row passes; interleaved columns per CTA of the
// column passes.
int row_pass_nseq(const Geometry& g);
template <typename T> int col_pass_width();
// Composite operator Phi^H Phi as a convolution, in real form: the image
// rows' half spectra (n x K/2 complex in B, entry 0 = X(0) + i X(K/2)).
// Forward row pass (prologue, zero-padding, row FFT of row pairs):
// deapod: S applied to both rows (Phi), or null (the convolution form).
template <typename T>
void launch_row_fwd_h(const Geometry& g, const RowPro<T>& pro, const T* deapod, typename cplx_t<T>::type* B,
                      const typename cplx_t<T>::type* tw, cudaStream_t s);
// Column pass: forward column FFT, multiply by the real PSF spectrum khat
// ([K/2/cw][K][cw], then column K/2 as K values), inverse FFT, crop (in place).
template <typename T>
void launch_col_conv_h(const Geometry& g, typename cplx_t<T>::type* B, const T* khat,
                       const typename cplx_t<T>::type* tw, cudaStream_t s);
// Real-form column passes of Phi (half-spectrum rows B -> the full padded
// grid, mirrored columns included) and Phi^H (padded accumulator Q -> the
// half-spectrum rows of its Hermitian part).
template <typename T>
void launch_col_fwd_h(const Geometry& g, const typename cplx_t<T>::type* B, typename cplx_t<T>::type* Pg,
                      const typename cplx_t<T>::type* tw, cudaStream_t s);
template <typename T>
void launch_col_inv_h(const Geometry& g, const typename cplx_t<T>::type* Q, typename cplx_t<T>::type* B,
                      const typename cplx_t<T>::type* tw, cudaStream_t s);
// Inverse row pass with the row epilogue (deapod: S^T, or null); returns the
// number of partial sums.
template <typename T>
int launch_row_inv_h(const Geometry& g, const typename cplx_t<T>::type* B, const T* deapod, const RowEp<T>& ep,
                     const typename cplx_t<T>::type* tw, cudaStream_t s);
// Batched real-form passes: `count` instances of the grid side g.K (image
// sides 64..1024), one launch, arguments from a device table (instance =
// blockIdx.y); every instance has g's launch shape.
template <typename T> void launch_row_fwd_h_batch(const Geometry& g, const RowFwdArgs<T>* tab, int count, cudaStream_t s);
template <typename T> void launch_col_conv_h_batch(const Geometry& g, const ColConvArgs<T>* tab, int count, cudaStream_t s);
template <typename T> void launch_col_fwd_h_batch(const Geometry& g, const ColFwdArgs<T>* tab, int count, cudaStream_t s);
template <typename T> void launch_col_inv_h_batch(const Geometry& g, const ColInvArgs<T>* tab, int count, cudaStream_t s);
template <typename T> void launch_row_inv_h_batch(const Geometry& g, const RowInvArgs<T>* tab, int count, cudaStream_t s);
// Real spectrum of the convolution kernel from the PSF image (2n x 2n real,
// pixel offsets [-n, n)^2): circulant embedding on the K = 2n grid, forward
// FFT, scaled by 1/K^2, columns [0, K/2] stored in launch_col_conv_h's layout
// (K/2 * K + K values).  X: K x K scratch.
template <typename T>
void build_psf_spectrum(const T* psf, int n, T* khat, typename cplx_t<T>::type* X,
                        const typename cplx_t<T>::type* tw, cudaStream_t s);
// In-place 2D FFT of a K x K complex array (dir -1 forward, +1 inverse, unnormalised).
template <typename T>
void launch_fft2_plain(int K, typename cplx_t<T>::type* X, const typename cplx_t<T>::type* tw, int dir,
                       cudaStream_t s);

template <typename T>
void launch_degrid(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items,
                   const Pos<T>* pos, const int* perm, const KbPoly<T>& kb, const DegridEp<typename cplx_t<T>::type>& ep,
                   int* err, cudaStream_t s);
template <typename T>
void launch_grid(const Geometry& g, const WorkItem* items, int n_items, const Pos<T>* pos, const int* perm,
                 const KbPoly<T>& kb, const GridPro<typename cplx_t<T>::type>& pro, typename cplx_t<T>::type* Q,
                 cudaStream_t s);
// Batched: `count` instances (their tiles may differ), one launch; the grid
// covers the largest instance's items (max_items) and the rest exit early.
template <typename T>
void launch_degrid_batch(const DegridArgs<T>* tab, int count, int max_items, int max_tb, const KbPoly<T>& kb,
                         cudaStream_t s);
template <typename T>
void launch_grid_batch(const GridArgs<T>* tab, int count, int max_items, int max_tb, const KbPoly<T>& kb,
                       cudaStream_t s);
template <typename T>
void launch_gram(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items, const Pos<T>* pos,
                 const KbPoly<T>& kb, typename cplx_t<T>::type* Q, int* err, cudaStream_t s);

// Stream-ordered memory for set-up temporaries (binning scratch, the PSF
// operator and its buffers): one pool per device that keeps up to
// kSetupPoolKeep bytes of released memory mapped, so that repeated operator
// creations reuse it instead of mapping new memory each time.
constexpr uint64_t kSetupPoolKeep = uint64_t(1) << 30;
cudaError_t setup_alloc(void** p, size_t bytes, cudaStream_t s);
template <typename U> cudaError_t setup_alloc(U** p, size_t bytes, cudaStream_t s) {
  return setup_alloc(reinterpret_cast<void**>(p), bytes, s);
}

// uv binning (once per operator).  Fills pos/perm and returns the work list.
// With R > 1 visibility blocks (device int32 block index per visibility, in
// caller order), visibilities are binned by (block, tile, cell) and every work
// item lies in one block (its `pad` field).
// Positions for the grid of twice the resolution of a binning of the Kc grid
// (fine tiles TB = 2 x the coarse tiles): the coarse items and order serve.
template <typename T>
void launch_encode_x2(const double* uv, const int* perm, int64_t M, int Kc, int TB, Pos<T>* pos, cudaStream_t s);
// items_pool: allocate the work list from this pool on `s` (else cudaMalloc).
template <typename T>
int build_bins(const double* uv, int64_t M, const Geometry& g, int chunk, Pos<T>* pos, int* perm,
               WorkItem** items_out, int* n_items_out, cudaStream_t s, const int* blocks = nullptr, int R = 1,
               cudaMemPool_t items_pool = nullptr);

// SARA dictionary.
template <typename T>
struct SaraPlan {
  int n, levels;
  T* s0;   // [8][(n/2)^2] scratch bands
  T* s1;
  T* cs;   // [9][n][n] scratch coefficients (prox output)
  DbFilters<T> f;
  // selected bases (sara_select): Dirac in slot 0 when dirac, then the nf
  // Daubechies filters fid[0..nf) (K - 1, increasing); scale = 1/sqrt(nbases)
  int dirac, nf, nbases;
  int fid[kMaxDb];
  T scale;
};
// Bases of the dictionary: bit 0 Dirac, bit K DbK (K = 1..8).
constexpr unsigned kSaraAll = 0x1FFu;
// Select the bases of `mask`; returns their number, or -1 for an invalid mask.
template <typename T> int sara_select(SaraPlan<T>& P, unsigned mask);
// Psi^H x (plain), c is [nbases][n][n].
template <typename T> void sara_analysis(const SaraPlan<T>& P, const T* x, T* c, cudaStream_t s);
// Psi c (plain).
template <typename T> void sara_synthesis(const SaraPlan<T>& P, const T* c, T* x, cudaStream_t s);

// SDMM l1 block fused with the analysis: v = Psi^H xh + z1; r = soft(v, gamma w);
// z1 = v - r; cs = 2r - v; objective partials sum w |Psi^H xh|.
template <typename T>
struct L1Block {
  T* z1;
  const T* w;      // may be null (w = 1)
  double gamma;
  double* partials;  // per-CTA partial objective, laid out by launch
};
// Returns number of objective partials written.
template <typename T>
int sara_analysis_prox(const SaraPlan<T>& P, const T* xh, const L1Block<T>& b, cudaStream_t s);
// x1 = Psi cs, then positivity block fused in the final level:
// v2 = xh + z2; r2 = max(v2, 0); z2 = v2 - r2; xs = x1 + 2 r2 - v2.
template <typename T>
void sara_synthesis_pos(const SaraPlan<T>& P, const T* xh, T* z2, T* xs, cudaStream_t s);
int sara_partials_capacity(int n, int levels);

// Batched SDMM blocks 1 and 2 (sara.cu): instances of one image side,
// wavelet levels and dictionary, every analysis / synthesis launch covering
// all of them.  Per instance: its plan (bands, filters, prox output cs), x_hat,
// z_1, the weights, gamma, its objective partials, z_2 and the output xs.
template <typename T> struct SaraBatchInst {
  const SaraPlan<T>* P;
  const T* xh;
  T* z1;
  const T* w;
  double gamma;
  double* partials;
  T* z2;
  T* xs;
};
template <typename T> struct SaraBatch;
// Builds the device argument tables; *np receives the objective partials
// each instance writes.
// pool: take the tables from this stream-ordered pool on `s` (else cudaMalloc).
template <typename T>
int sara_batch_create(const std::vector<SaraBatchInst<T>>& in, SaraBatch<T>** out, int* np,
                      cudaMemPool_t pool = nullptr, cudaStream_t s = nullptr);
template <typename T> void sara_batch_launch(const SaraBatch<T>* b, cudaStream_t s);
template <typename T> void sara_batch_destroy(SaraBatch<T>* b);
// Objective partials the fused analysis of P writes.
template <typename T> int sara_prox_partials(const SaraPlan<T>& P);

// TV prior (Section 4's TV / RWTV): the SDMM TV block with the positivity
// block fused into its epilogue (tv.cu).  v: n x n scratch; qa, qb: the
// dual's two buffers (2 n^2 each; the dual enters and leaves in qa).
template <typename T> struct TvBlock {
  int n, iters;
  double gamma;
  const T* xh;
  T* z1;
  T* z2;
  const T* w;  // may be null (w = 1)
  T* v;
  T* qa;
  T* qb;
  T* xs;
  double* partials;  // per-CTA objective partials (tv_partials(n) of them)
};
template <typename T> int tv_block(const TvBlock<T>& b, cudaStream_t s);
// |grad x| per pixel (forward differences, zero past the last row / column).
template <typename T> void tv_magnitude(const T* x, T* out, int n, cudaStream_t s);
int tv_partials(int n);

}  // namespace purify
