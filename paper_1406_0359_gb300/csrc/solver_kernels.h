// Vector kernels and device scalars of the SDMM solver.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

namespace purify {

// Device scalar slots (double[kNumScalars]).
enum ScalarSlot : int {
  S_RR = 0, S_ALPHA, S_BETA, S_PAP, S_BALLSCALE, S_BALLNORM, S_RESID, S_OBJ,
  S_LAMBDA, S_INVNORM, S_MEAN, S_STD, S_MAXABS, S_FEAS,
  S_CG0,  // S_CG0 .. S_CG0 + 4: a CG step's five inner products, accumulated across CTAs (zero between steps)
  kNumScalars = S_CG0 + 5
};
enum FinOp : int { FIN_OBJ = 0, FIN_NORM, FIN_MEAN, FIN_VAR };
enum RedOp : int { RED_SQ = 0, RED_SUM, RED_VAR, RED_MAXABS };

int vec_blocks(size_t N);
// x += sc[idx] p; N a multiple of 4, both arrays 16-byte aligned.
template <typename T> void launch_axpy(T* x, const T* p, const double* sc, int idx, size_t N, cudaStream_t s);
// Merge na partials (Acc<T> values in double-sized slots) and apply `op`.
template <typename T> void launch_finalize(const double* pa, int na, int op, double arg, double* sc, cudaStream_t s);
template <typename T>
int launch_reduce(const T* v, size_t N, int op, const double* sc, double* partials, cudaStream_t s);
void launch_max_partials(const double* p, int np, double* sc, cudaStream_t s);
// Ball scalars per visibility block; items_as_int points at the WorkItem array
// (four ints per item, the block in the fourth).  With R = 1, cpart (2 x
// kFinCtas doubles) and a zeroed ticket, the merge runs on up to kFinCtas
// CTAs in two levels; otherwise on one CTA.
constexpr int kFinCtas = 64;
template <typename T>
void launch_finalize_blocks(const double* part0, const double* part1, const int* items_as_int, int n_items, int R,
                            double nu, const double* eps_b, double* scale_b, double* sc, double* cpart,
                            unsigned int* ticket, cudaStream_t s);
template <typename T> void launch_reweight(T* w, size_t N, double delta, cudaStream_t s);
template <typename T> void launch_fill(T* v, size_t N, T val, cudaStream_t s);
template <typename T> void launch_scale(T* v, size_t N, const double* sc, int idx, double mul, cudaStream_t s);
template <typename C> void launch_gather(const C* src, const int* perm, size_t M, C* dst, cudaStream_t s);
// Batched vector steps of instances of one size (argument tables in device
// memory; instance = blockIdx.y, one grid for all).
template <typename T> struct AxpyArgs { T* x; const T* p; const double* sc; int idx; size_t N; };
template <typename T> void launch_axpy_batch(const AxpyArgs<T>* tab, int count, size_t N, cudaStream_t s);
struct FinArgs { const double* pa; int na; int op; double arg; double* sc; };
template <typename T> void launch_finalize_batch(const FinArgs* tab, int count, cudaStream_t s);
struct Ball1Args {
  const double* part0;
  const double* part1;
  int n_items;
  double nu;
  const double* eps_b;
  double* scale_b;
  double* sc;
  double* cpart;
  unsigned int* ticket;
};
// kFinCtas CTAs per instance (the two-level merge of the R = 1 ball scalars).
template <typename T> void launch_finalize_ball1_batch(const Ball1Args* tab, int count, cudaStream_t s);
struct ZeroArgs { void* p; size_t bytes; };  // bytes a multiple of 16
void launch_zero_batch(const ZeroArgs* tab, int count, size_t max_bytes, cudaStream_t s);

// Device flag set when any of the n values is not finite (NaN or infinity).
template <typename T> void launch_check_finite(const T* v, size_t n, int* flag, cudaStream_t s);

}  // namespace purify
