// Learned preconditioner of the pinned-Laplacian block solves (see mlp.cu).
#pragma once

#include "internal.cuh"

namespace sbha {

constexpr int kMlpHidden = 64;
constexpr int kMlpFeatures = 6;
constexpr int kMlpParams =
    kMlpHidden * kMlpFeatures + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;
constexpr int kPrecondMaxTrainCols = 512;
constexpr int kPilotCols = 32;       // columns the plain solver solves before the network trains on them
constexpr double kPilotRtol = 1e-3;  // their tolerance: training pairs need no more

// Device-side checks and conversions for the preconditioner entry point.
void check_rowptr(Ctx& c, int64_t m, const int32_t* rowptr);  // rows non-decreasing, else SBHA_EINVAL
void to_float(Ctx& c, int64_t n, const double* x, float* y);
// row-major m x ncols into block layout with ceil(ncols/32) blocks, zero-padded
void rows_to_blocks(Ctx& c, int64_t m, int ncols, const double* B, double* out);

// Mean-squared-error loss and its gradient for N samples (X: N x 6, T: N; FP32 device arrays).
void mlp_gradient(Ctx& c, int64_t N, const float* X, const float* T, const float* params, float* grad, double* loss);

// M^{-1} = G^T G for an SPD matrix A with a symmetric CSR pattern (sorted columns, diagonal
// present).  G has A's pattern; its entries come from a small network evaluated on scale-free
// features of each entry, G_ij = (delta_ij + y(f_ij)) / sqrt(A_ii), so that the untrained
// network (last layer zero) is the Jacobi preconditioner D^{-1}.
struct LearnedPrecond {
  Ctx& c;
  int64_t m = 0, nnz = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;   // A (FP64)
  const float* val32 = nullptr;  // A (FP32)
  float* feat = nullptr;         // [nnz][6]
  int32_t* erow = nullptr;       // [nnz] row of each entry
  int32_t* tpos = nullptr;       // [nnz] position of the transposed entry
  double* sc = nullptr;          // [m] 1 / sqrt(A_ii)
  float* g32 = nullptr;          // G, FP32, A's CSR order
  float* gt32 = nullptr;         // G^T in A's CSR order (row j holds G_ij)
  double* g64 = nullptr;
  double* gt64 = nullptr;
  float* params = nullptr;
  bool trained = false;
  int64_t train_entries = 0;  // entries of G the last training touched

  LearnedPrecond(Ctx& ctx, int64_t m, int64_t nnz, const int32_t* rowptr, const int32_t* col, const double* val,
                 const float* val32);
  // Loss  sum_c w_c ||A (G^T G b_c - x_c)||^2,  w_c = 1 / (ncols ||b_c||^2),  over ncols pairs of
  // right-hand sides B and solutions X of A X = B (block layout: column c of row u at
  // ((c/32) m + u) 32 + c%32, FP64; X nullable: then A x_c = b_c is taken as exact), and its
  // gradient with respect to the network parameters.
  void loss_grad(const double* B, const double* X, int ncols, const float* p, float* grad, double* loss);
  // Full-batch Adam from the Jacobi start on the same loss; fills G (all precisions) and returns
  // true when the loss fell below half its starting value.
  bool train(const double* B, const double* X, int ncols, int epochs, float lr, double* loss_first,
             double* loss_last);
  // G and G^T from the current parameters (all entries)
  void assemble();
  // Overwrites G and G^T (all precisions) with NaN: host-side fault injection for the fallback tests.
  void poison();
};

}  // namespace sbha
