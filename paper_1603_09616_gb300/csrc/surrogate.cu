// Learned surrogate for the energy-integrated local outputs (local charge q_j,
// local energy E_j): a per-orbital environment descriptor and a small MLP
// (64 -> 128 -> 128 -> 128 -> 2, GELU, BF16 weights, FP32 accumulation) with
// forward, backward and Adam kernels.  The shifted solver produces the training
// labels and stays the judge (see the Python driver).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/gbgreen_surrogate.h"
#include "gb_internal.h"
#include "kernels.cuh"

namespace gb {
const gbk::DevMat* devmat_of(const gb_matrix* m);  // the matrix's device view (solver.cu)
}

namespace {

constexpr int kDesc = 64;
constexpr float kRc = 0.5f;       // nm, descriptor cutoff
constexpr float kRbfW = 0.03f;    // nm, radial Gaussian width

__device__ __forceinline__ float cutoff_fn(float r) { return r < kRc ? 0.5f * (cospif(r / kRc) + 1.0f) : 0.0f; }

// One thread per orbital j.  Features (all from the pattern row j, whose
// orbitals belong to the atoms within the interaction cutoff):
//   0-15  radial Gaussians (centres 0.1..0.5 nm) over carbon neighbour atoms
//   16-31 the same over hydrogen neighbour atoms
//   32-39 angular: per radial shell (4 shells of 0.125 nm) the squared norm of
//         the cutoff-weighted dipole (l = 1) and traceless quadrupole (l = 2)
//         of the neighbour directions
//   40-41 own species one-hot, 42-45 orbital slot one-hot
//   46 H_jj, 47 S_jj
//   48-55 neighbour onsite energies H_ii in 8 Gaussian bins on [-3, 3] eV,
//         weighted by H_ji^2
//   56 sum H_ji^2, 57 sum S_ji^2, 58 sum H_ji S_ji, 59 sum H_ji^2 H_ii,
//   60 sum |H_ji|, 61 |R_j| / 100, 62 sum S_ji H_ii (all over i != j), 63 = 1
__global__ void descriptor_kernel(const gbk::DevMat m, const float* __restrict__ pos, const int* __restrict__ orb_atom,
                                  const int* __restrict__ atom_first, const int* __restrict__ species,
                                  float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m.n) return;
  float f[kDesc];
#pragma unroll
  for (int k = 0; k < kDesc; ++k) f[k] = 0.f;
  const int a = orb_atom[j];
  const float ax = pos[3 * a], ay = pos[3 * a + 1], az = pos[3 * a + 2];
  float dip[4][3] = {};
  float quad[4][6] = {};
  const int lo = m.row_ptr[j], hi = m.row_ptr[j + 1];
  for (int e = lo; e < hi; ++e) {
    const int i = m.col_idx[e];
    const int b = orb_atom[i];
    const double hji = m.h_val[e], sji = m.s_val[e];
    if (i == j) {
      f[46] = (float)hji;
      f[47] = (float)sji;
      continue;
    }
    // H_ii: diagonal entry of row i (binary search in the sorted row)
    int l0 = m.row_ptr[i], l1 = m.row_ptr[i + 1] - 1;
    while (l0 < l1) {
      const int mid = (l0 + l1) >> 1;
      if (m.col_idx[mid] < i) l0 = mid + 1;
      else l1 = mid;
    }
    const float hii = (float)m.h_val[l0];
    const float h2 = (float)(hji * hji);
    for (int t = 0; t < 8; ++t) {
      const float c = -3.0f + 6.0f * t / 7.0f, d = (hii - c) / 0.75f;
      f[48 + t] += h2 * __expf(-d * d);
    }
    f[56] += h2;
    f[57] += (float)(sji * sji);
    f[58] += (float)(hji * sji);
    f[59] += h2 * hii;
    f[60] += fabsf((float)hji);
    f[62] += (float)sji * hii;
    if (b == a || i != atom_first[b]) continue;  // geometric part: each neighbour atom once
    const float dx = pos[3 * b] - ax, dy = pos[3 * b + 1] - ay, dz = pos[3 * b + 2] - az;
    const float r = sqrtf(dx * dx + dy * dy + dz * dz);
    if (!(r > 1e-6f) || r >= kRc) continue;
    const float w = cutoff_fn(r);
    const int sb = species[b] ? 16 : 0;
    for (int t = 0; t < 16; ++t) {
      const float mu = 0.1f + 0.4f * t / 15.0f, d = (r - mu) / kRbfW;
      f[sb + t] += w * __expf(-d * d);
    }
    const int sh = min(3, (int)(r / (kRc / 4)));
    const float ux = dx / r, uy = dy / r, uz = dz / r;
    dip[sh][0] += w * ux;
    dip[sh][1] += w * uy;
    dip[sh][2] += w * uz;
    quad[sh][0] += w * (ux * ux - 1.0f / 3);
    quad[sh][1] += w * (uy * uy - 1.0f / 3);
    quad[sh][2] += w * (uz * uz - 1.0f / 3);
    quad[sh][3] += w * ux * uy;
    quad[sh][4] += w * ux * uz;
    quad[sh][5] += w * uy * uz;
  }
  for (int s = 0; s < 4; ++s) {
    f[32 + 2 * s] = dip[s][0] * dip[s][0] + dip[s][1] * dip[s][1] + dip[s][2] * dip[s][2];
    f[33 + 2 * s] = quad[s][0] * quad[s][0] + quad[s][1] * quad[s][1] + quad[s][2] * quad[s][2] +
                    2.f * (quad[s][3] * quad[s][3] + quad[s][4] * quad[s][4] + quad[s][5] * quad[s][5]);
  }
  f[40 + (species[a] ? 1 : 0)] = 1.f;
  f[42 + min(3, j - atom_first[a])] = 1.f;
  f[61] = (hi - lo) / 100.0f;
  f[63] = 1.f;
  float* o = out + (size_t)j * kDesc;
#pragma unroll
  for (int k = 0; k < kDesc; ++k) o[k] = f[k];
}

// ------------------------------------------------------------ MLP kernels
__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
  const float cdf = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * __expf(-0.5f * x * x);
  return cdf + x * pdf;
}

constexpr int TILE = 32;

// Y[B x out] = X[B x in] W^T + b, W stored [out x in] in BF16; pre-activation
// kept in P, activation (GELU or identity) in Y.  FP32 accumulation.
__global__ void dense_fwd(const float* __restrict__ X, const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                          int B, int nin, int nout, int act, float* __restrict__ P, float* __restrict__ Y) {
  __shared__ float xs[TILE][TILE + 1];
  __shared__ float ws[TILE][TILE + 1];
  const int row = blockIdx.y * TILE + threadIdx.y;  // sample
  const int col = blockIdx.x * TILE + threadIdx.x;  // output unit
  float acc = 0.f;
  for (int k0 = 0; k0 < nin; k0 += TILE) {
    const int kx = k0 + threadIdx.x;
    xs[threadIdx.y][threadIdx.x] = (row < B && kx < nin) ? X[(size_t)row * nin + kx] : 0.f;
    const int wo = blockIdx.x * TILE + threadIdx.y;  // output unit loaded by this thread row
    ws[threadIdx.y][threadIdx.x] = (wo < nout && kx < nin) ? __bfloat162float(W[(size_t)wo * nin + kx]) : 0.f;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TILE; ++k) acc = fmaf(xs[threadIdx.y][k], ws[threadIdx.x][k], acc);
    __syncthreads();
  }
  if (row < B && col < nout) {
    const float p = acc + bias[col];
    P[(size_t)row * nout + col] = p;
    Y[(size_t)row * nout + col] = act ? gelu(p) : p;
  }
}

// G = dY * act'(P) (in place into G), dX[B x in] = G W (BF16 weights)
__global__ void dense_bwd_x(const float* __restrict__ G, const __nv_bfloat16* __restrict__ W, int B, int nin, int nout,
                            float* __restrict__ dX) {
  __shared__ float gs[TILE][TILE + 1];
  __shared__ float ws[TILE][TILE + 1];
  const int row = blockIdx.y * TILE + threadIdx.y;  // sample
  const int col = blockIdx.x * TILE + threadIdx.x;  // input unit
  float acc = 0.f;
  for (int o0 = 0; o0 < nout; o0 += TILE) {
    const int ox = o0 + threadIdx.x;
    gs[threadIdx.y][threadIdx.x] = (row < B && ox < nout) ? G[(size_t)row * nout + ox] : 0.f;
    const int oy = o0 + threadIdx.y;
    const int ic = blockIdx.x * TILE + threadIdx.x;
    ws[threadIdx.y][threadIdx.x] = (oy < nout && ic < nin) ? __bfloat162float(W[(size_t)oy * nin + ic]) : 0.f;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TILE; ++k) acc = fmaf(gs[threadIdx.y][k], ws[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (row < B && col < nin) dX[(size_t)row * nin + col] = acc;
}

__global__ void act_grad(float* __restrict__ G, const float* __restrict__ P, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    G[i] *= gelu_grad(P[i]);
}

// dW[out x in] = G^T X (sum over the batch), db = column sums of G; one block
// per (out tile, in tile), batch looped in fixed order (deterministic).
__global__ void dense_bwd_w(const float* __restrict__ G, const float* __restrict__ X, int B, int nin, int nout,
                            float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float gs[TILE][TILE + 1];
  __shared__ float xs[TILE][TILE + 1];
  const int o = blockIdx.y * TILE + threadIdx.y;
  const int i = blockIdx.x * TILE + threadIdx.x;
  float acc = 0.f, accb = 0.f;
  for (int s0 = 0; s0 < B; s0 += TILE) {
    const int sg = s0 + threadIdx.x;
    const int oy = blockIdx.y * TILE + threadIdx.y;
    gs[threadIdx.y][threadIdx.x] = (sg < B && oy < nout) ? G[(size_t)sg * nout + oy] : 0.f;
    const int sx = s0 + threadIdx.y;
    xs[threadIdx.y][threadIdx.x] = (sx < B && i < nin) ? X[(size_t)sx * nin + i] : 0.f;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < TILE; ++k) {
      acc = fmaf(gs[threadIdx.y][k], xs[k][threadIdx.x], acc);
      accb += gs[threadIdx.y][k];
    }
    __syncthreads();
  }
  if (o < nout && i < nin) dW[(size_t)o * nin + i] = acc;
  if (o < nout && blockIdx.x == 0 && threadIdx.x == 0) db[o] = accb;
}

__global__ void mse_grad(const float* __restrict__ Y, const float* __restrict__ T, size_t n, float scale,
                         float* __restrict__ dY, float* __restrict__ partial) {
  __shared__ float red[256];
  float s = 0.f;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = 2.0f * scale * d;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0] * scale;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            __nv_bfloat16* __restrict__ wb, size_t n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void affine_cols(float* __restrict__ X, size_t n, int cols, const float* __restrict__ scale,
                            const float* __restrict__ shift) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % cols);
    X[i] = fmaf(X[i], scale[c], shift[c]);
  }
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

}  // namespace

extern "C" {

gb_status gb_descriptors(const gb_matrix* m, int32_t n_atoms, const float* pos, const int32_t* orb_atom,
                         const int32_t* atom_first, const int32_t* species, float* out, void* stream) {
  gb::clear_error();
  if (!m || !pos || !orb_atom || !atom_first || !species || !out || n_atoms < 1)
    return gb::fail(GB_EINVAL, "gb_descriptors: NULL argument or no atoms");
  const gbk::DevMat* dm = gb::devmat_of(m);
  const int threads = 128;
  descriptor_kernel<<<(dm->n + threads - 1) / threads, threads, 0, static_cast<cudaStream_t>(stream)>>>(
      *dm, pos, orb_atom, atom_first, species, out);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "descriptor kernel: %s", cudaGetErrorString(e));
  return GB_OK;
}

size_t gb_mlp_workspace_size(const gb_mlp* net, int32_t batch) {
  if (!net || batch < 1) return 0;
  // per layer: pre-activation and activation [batch x width]; plus two gradient buffers
  size_t tot = 0;
  for (int l = 0; l < GB_MLP_LAYERS; ++l) tot += 2 * (size_t)batch * net->dims[l + 1];
  tot += 2 * (size_t)batch * GB_MLP_MAXW;
  tot += 152 * 16;  // loss partials
  return tot * sizeof(float);
}

static gb_status check_net(const gb_mlp* net) {
  if (!net) return gb::fail(GB_EINVAL, "net is NULL");
  for (int l = 0; l < GB_MLP_LAYERS; ++l) {
    if (net->dims[l] < 1 || net->dims[l] > GB_MLP_MAXW || net->dims[l + 1] < 1 || net->dims[l + 1] > GB_MLP_MAXW)
      return gb::fail(GB_EINVAL, "layer widths must be in [1, %d]", GB_MLP_MAXW);
    if (!net->w[l] || !net->w_bf16[l] || !net->b[l]) return gb::fail(GB_EINVAL, "layer %d has NULL weights", l);
  }
  return GB_OK;
}

gb_status gb_mlp_forward(const gb_mlp* net, const float* X, int32_t batch, float* Y, float* ws, size_t ws_bytes,
                         void* stream) {
  gb::clear_error();
  gb_status st = check_net(net);
  if (st != GB_OK) return st;
  if (!X || !Y || !ws || batch < 1) return gb::fail(GB_EINVAL, "gb_mlp_forward: bad arguments");
  if (ws_bytes < gb_mlp_workspace_size(net, batch)) return gb::fail(GB_ENOMEM, "MLP workspace too small");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float* in = X;
  float* base = ws;
  for (int l = 0; l < GB_MLP_LAYERS; ++l) {
    const int nin = net->dims[l], nout = net->dims[l + 1];
    float* P = base;
    float* A = base + (size_t)batch * nout;
    base = A + (size_t)batch * nout;
    const bool last = l == GB_MLP_LAYERS - 1;
    dim3 blk(TILE, TILE), grd((nout + TILE - 1) / TILE, (batch + TILE - 1) / TILE);
    dense_fwd<<<grd, blk, 0, s>>>(in, reinterpret_cast<const __nv_bfloat16*>(net->w_bf16[l]), net->b[l], batch, nin,
                                  nout, last ? 0 : 1, P, last ? Y : A);
    in = A;
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "MLP forward: %s", cudaGetErrorString(e));
  return GB_OK;
}

gb_status gb_mlp_backward(const gb_mlp* net, const float* X, const float* dY, int32_t batch, float* ws,
                          size_t ws_bytes, void* stream) {
  gb::clear_error();
  gb_status st = check_net(net);
  if (st != GB_OK) return st;
  if (!X || !dY || !ws || batch < 1) return gb::fail(GB_EINVAL, "gb_mlp_backward: bad arguments");
  if (ws_bytes < gb_mlp_workspace_size(net, batch)) return gb::fail(GB_ENOMEM, "MLP workspace too small");
  for (int l = 0; l < GB_MLP_LAYERS; ++l)
    if (!net->gw[l] || !net->gb[l]) return gb::fail(GB_EINVAL, "layer %d has NULL gradient buffers", l);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* P[GB_MLP_LAYERS];
  float* A[GB_MLP_LAYERS];
  float* base = ws;
  for (int l = 0; l < GB_MLP_LAYERS; ++l) {
    P[l] = base;
    A[l] = base + (size_t)batch * net->dims[l + 1];
    base = A[l] + (size_t)batch * net->dims[l + 1];
  }
  float* g0 = base;
  float* g1 = base + (size_t)batch * GB_MLP_MAXW;
  cudaMemcpyAsync(g0, dY, sizeof(float) * (size_t)batch * net->dims[GB_MLP_LAYERS], cudaMemcpyDeviceToDevice, s);
  for (int l = GB_MLP_LAYERS - 1; l >= 0; --l) {
    const int nin = net->dims[l], nout = net->dims[l + 1];
    if (l != GB_MLP_LAYERS - 1) {
      const size_t n = (size_t)batch * nout;
      act_grad<<<grid_for(n), 256, 0, s>>>(g0, P[l], n);
    }
    const float* xin = l == 0 ? X : A[l - 1];
    dim3 blk(TILE, TILE);
    dense_bwd_w<<<dim3((nin + TILE - 1) / TILE, (nout + TILE - 1) / TILE), blk, 0, s>>>(g0, xin, batch, nin, nout,
                                                                                          net->gw[l], net->gb[l]);
    if (l > 0) {
      dense_bwd_x<<<dim3((nin + TILE - 1) / TILE, (batch + TILE - 1) / TILE), blk, 0, s>>>(
          g0, reinterpret_cast<const __nv_bfloat16*>(net->w_bf16[l]), batch, nin, nout, g1);
      float* t = g0;
      g0 = g1;
      g1 = t;
    }
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "MLP backward: %s", cudaGetErrorString(e));
  return GB_OK;
}

gb_status gb_mse_grad(const float* Y, const float* T, int32_t batch, int32_t nout, float* dY, float* partial,
                      int32_t* npartial, void* stream) {
  gb::clear_error();
  if (!Y || !T || !dY || !partial || !npartial || batch < 1 || nout < 1) return gb::fail(GB_EINVAL, "gb_mse_grad: bad arguments");
  const size_t n = (size_t)batch * nout;
  const int g = grid_for(n);
  mse_grad<<<g, 256, 0, static_cast<cudaStream_t>(stream)>>>(Y, T, n, 1.0f / (float)n, dY, partial);
  *npartial = g;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "mse kernel: %s", cudaGetErrorString(e));
  return GB_OK;
}

gb_status gb_mlp_adam(gb_mlp* net, float lr, float beta1, float beta2, float eps, int32_t step, void* stream) {
  gb::clear_error();
  gb_status st = check_net(net);
  if (st != GB_OK) return st;
  if (step < 1) return gb::fail(GB_EINVAL, "Adam step counts from 1");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  for (int l = 0; l < GB_MLP_LAYERS; ++l) {
    if (!net->mw[l] || !net->vw[l] || !net->mb[l] || !net->vb[l]) return gb::fail(GB_EINVAL, "Adam moments are NULL");
    const size_t nw = (size_t)net->dims[l] * net->dims[l + 1], nb = net->dims[l + 1];
    adam_kernel<<<grid_for(nw), 256, 0, s>>>(net->w[l], net->gw[l], net->mw[l], net->vw[l],
                                             reinterpret_cast<__nv_bfloat16*>(net->w_bf16[l]), nw, lr, beta1, beta2,
                                             eps, c1, c2);
    adam_kernel<<<grid_for(nb), 256, 0, s>>>(net->b[l], net->gb[l], net->mb[l], net->vb[l], nullptr, nb, lr, beta1,
                                             beta2, eps, c1, c2);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "Adam kernel: %s", cudaGetErrorString(e));
  return GB_OK;
}

gb_status gb_affine_cols(float* X, int32_t rows, int32_t cols, const float* scale, const float* shift,
                         void* stream) {
  gb::clear_error();
  if (!X || !scale || !shift || rows < 0 || cols < 1) return gb::fail(GB_EINVAL, "gb_affine_cols: bad arguments");
  const size_t n = (size_t)rows * cols;
  if (n == 0) return GB_OK;
  affine_cols<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(X, n, cols, scale, shift);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "affine kernel: %s", cudaGetErrorString(e));
  return GB_OK;
}

gb_status gb_mlp_sync_bf16(gb_mlp* net, void* stream) {
  gb::clear_error();
  gb_status st = check_net(net);
  if (st != GB_OK) return st;
  for (int l = 0; l < GB_MLP_LAYERS; ++l) {
    const size_t nw = (size_t)net->dims[l] * net->dims[l + 1];
    to_bf16<<<grid_for(nw), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        net->w[l], reinterpret_cast<__nv_bfloat16*>(net->w_bf16[l]), nw);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return gb::fail(GB_ECUDA, "bf16 copy: %s", cudaGetErrorString(e));
  return GB_OK;
}

}  // extern "C"
