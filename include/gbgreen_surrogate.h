/*
 * gbgreen_surrogate.h — C ABI of the learned surrogate for local outputs.
 *
 * The energy-integrated local outputs of the shifted Green's-function solver
 * (local charge q_j = sum_i rho_ij S_ij and local energy E_j = sum_i rho_ij
 * H_ij) depend mostly on each orbital's neighbourhood.  A small MLP trained on
 * solver-generated labels predicts them from a per-orbital environment
 * descriptor; the solver remains the judge (re-solving a sample and a
 * fallback set).  The paper motivates data-driven analysis of the large
 * simulation outputs (Summary and future outlook) but gives no model; this is
 * the library's own.
 *
 * All pointers are device pointers (caller-owned) unless noted; every call is
 * asynchronous on `stream`.  Return values: gb_status from gbgreen.h.
 */
#ifndef GBGREEN_SURROGATE_H
#define GBGREEN_SURROGATE_H

#include "gbgreen.h"

#ifdef __cplusplus
extern "C" {
#endif

#define GB_DESC_DIM 64
#define GB_MLP_LAYERS 4
#define GB_MLP_MAXW 128

/*
 * gb_descriptors — 64 floats per orbital (row-major [n][64]) from the atom
 * positions (nm, [n_atoms][3] float), the orbital -> atom map ([n] int32),
 * the first orbital of every atom ([n_atoms + 1] int32), the species per atom
 * ([n_atoms] int32, 0 carbon, 1 hydrogen) and the rows of H and S in `m`.
 * Radial Gaussians (carbon and hydrogen neighbours), dipole and quadrupole
 * magnitudes of the neighbour directions per radial shell, species and
 * orbital-slot one-hots, H_jj, S_jj, and coupling-weighted statistics of the
 * neighbours' onsite energies (see the kernel's comment for the exact list).
 */
gb_status gb_descriptors(const gb_matrix* m, int32_t n_atoms, const float* pos, const int32_t* orb_atom,
                         const int32_t* atom_first, const int32_t* species, float* out, void* stream);

/*
 * The network: dims[0] -> dims[1] -> ... -> dims[GB_MLP_LAYERS] with GELU
 * after every layer but the last.  Layer l: FP32 master weights w[l]
 * [dims[l+1]][dims[l]] (row-major), BF16 copy w_bf16[l] (uint16 storage, the
 * copy the forward and backward products use), bias b[l] [dims[l+1]];
 * gradients gw, gb and Adam moments mw, vw, mb, vb of the same shapes.
 */
typedef struct {
  int32_t dims[GB_MLP_LAYERS + 1];
  float* w[GB_MLP_LAYERS];
  uint16_t* w_bf16[GB_MLP_LAYERS];
  float* b[GB_MLP_LAYERS];
  float* gw[GB_MLP_LAYERS];
  float* gb[GB_MLP_LAYERS];
  float* mw[GB_MLP_LAYERS];
  float* vw[GB_MLP_LAYERS];
  float* mb[GB_MLP_LAYERS];
  float* vb[GB_MLP_LAYERS];
} gb_mlp;

/* Bytes of activation workspace for a batch (forward and backward share it). */
size_t gb_mlp_workspace_size(const gb_mlp* net, int32_t batch);

/* Y [batch][dims[L]] = net(X [batch][dims[0]]); keeps the activations in ws. */
gb_status gb_mlp_forward(const gb_mlp* net, const float* X, int32_t batch, float* Y, float* ws, size_t ws_bytes,
                         void* stream);

/* Gradients of sum(dY * Y) into gw, gb; needs the activations of the forward
 * call on the same X with the same ws. */
gb_status gb_mlp_backward(const gb_mlp* net, const float* X, const float* dY, int32_t batch, float* ws,
                          size_t ws_bytes, void* stream);

/* Mean-squared-error gradient dY = 2 (Y - T) / (batch * nout); partial sums of
 * the loss go to partial[0 .. *npartial) (caller sums them; the host int
 * *npartial is set by the call, at most 2432 entries). */
gb_status gb_mse_grad(const float* Y, const float* T, int32_t batch, int32_t nout, float* dY, float* partial,
                      int32_t* npartial, void* stream);

/* One Adam step (bias-corrected, step >= 1) on every layer; refreshes w_bf16. */
gb_status gb_mlp_adam(gb_mlp* net, float lr, float beta1, float beta2, float eps, int32_t step, void* stream);

/* X[r][c] = X[r][c] * scale[c] + shift[c] for a row-major [rows][cols] float
 * array (feature standardisation and its inverse). */
gb_status gb_affine_cols(float* X, int32_t rows, int32_t cols, const float* scale, const float* shift,
                         void* stream);

/* Round the FP32 master weights into the BF16 copies. */
gb_status gb_mlp_sync_bf16(gb_mlp* net, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GBGREEN_SURROGATE_H */
