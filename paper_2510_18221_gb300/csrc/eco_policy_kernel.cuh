// eco_policy_kernel.cuh -- the policy kernel template (internal).  Each
// precision's instances are compiled in their own translation unit
// (eco_policy_fp32.cu, eco_policy_bf16.cu, eco_policy_fp8.cu); eco_policy.cu
// holds the variant table and the launch.
//
// The policy phase of the step: observation gather
// (Sec. 3.2 "Sensors"), per-agent MLP D -> H -> H -> A with tanh hidden
// layers (Sec. 3.3), and Gumbel-max sampling of the action (Sec. 3.3:
// actions are sampled from a softmax over the logits).
//
// Every agent owns its weights, so the work is a batch of independent
// matrix-vector products bound by HBM reads of the weights (about 57 KB per
// agent in BF16 at 371 -> 64 -> 64 -> 9), not a dense contraction: tensor
// cores do not apply.  The kernel is warp-per-agent:
//   * the warp gathers the agent's k x k patch (3 or 4 channels) and scalars
//     into its own shared-memory row (one byte per cell: food / wall /
//     agent bits; RGB and terrain add the colour and resource reads);
//   * each lane streams 16-byte units of the agent's weight block with
//     non-allocating loads, UNROLL units in flight per lane; a warp load is
//     512 contiguous bytes;
//   * in the input-major layout a lane's units always hold the same group of
//     E outputs, so the lane accumulates E partial sums in FP32, and a
//     reduce-scatter over the lanes with the same group leaves each lane
//     H / 32 finished outputs;
//   * the head (A rows, output-major) reduces over small lane groups, and a
//     warp argmax of logit + Gumbel picks the action (ties to the lowest
//     action index).
// All floating-point reductions run in a fixed order, so results are
// bit-reproducible from run to run.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "eco_internal.cuh"
#include "eco_kernels.h"

namespace eco {

// Asynchronous prefetch of [p, p + bytes) into L2 (p and bytes multiples of
// 16), issued by one lane; it returns at once.
__device__ __forceinline__ void prefetch_l2(const void *p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint4 ldg_stream(const uint4 *p) {
  uint4 r;
  asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
      : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
      : "l"(p));
  return r;
}

// Two FP32 fused multiply-adds in one instruction (Blackwell's packed FP32
// pipe): a0 += w0 * x and a1 += w1 * x, each rounded once as by fmaf, so the
// results are bit-identical to two fmaf calls while the weight stream issues
// half as many FMA instructions.
__device__ __forceinline__ void ffma2(float &a0, float &a1, float w0, float w1, float x) {
  asm("{\n\t.reg .b64 pa, pw, px;\n\t"
      "mov.b64 pa, {%0, %1};\n\t"
      "mov.b64 pw, {%2, %3};\n\t"
      "mov.b64 px, {%4, %4};\n\t"
      "fma.rn.f32x2 pa, pw, px, pa;\n\t"
      "mov.b64 {%0, %1}, pa;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(w0), "f"(w1), "f"(x));
}

template <int PREC>
struct Unit;

template <>
struct Unit<PREC_FP32> {
  static constexpr int E = 4;
  __device__ __forceinline__ static void fma(float *acc, const uint4 &v, float x) {
    ffma2(acc[0], acc[1], __uint_as_float(v.x), __uint_as_float(v.y), x);
    ffma2(acc[2], acc[3], __uint_as_float(v.z), __uint_as_float(v.w), x);
  }
  __device__ __forceinline__ static float dot(const uint4 &v, const float *h) {
    const float4 a = *reinterpret_cast<const float4 *>(h);
    float s = __uint_as_float(v.x) * a.x;
    s = fmaf(__uint_as_float(v.y), a.y, s);
    s = fmaf(__uint_as_float(v.z), a.z, s);
    s = fmaf(__uint_as_float(v.w), a.w, s);
    return s;
  }
};

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

template <>
struct Unit<PREC_BF16> {
  static constexpr int E = 8;
  __device__ __forceinline__ static void fma(float *acc, const uint4 &v, float x) {
    ffma2(acc[0], acc[1], bf_lo(v.x), bf_hi(v.x), x);
    ffma2(acc[2], acc[3], bf_lo(v.y), bf_hi(v.y), x);
    ffma2(acc[4], acc[5], bf_lo(v.z), bf_hi(v.z), x);
    ffma2(acc[6], acc[7], bf_lo(v.w), bf_hi(v.w), x);
  }
  __device__ __forceinline__ static float dot(const uint4 &v, const float *h) {
    const float4 a = *reinterpret_cast<const float4 *>(h);
    const float4 b = *reinterpret_cast<const float4 *>(h + 4);
    float s = bf_lo(v.x) * a.x;
    s = fmaf(bf_hi(v.x), a.y, s);
    s = fmaf(bf_lo(v.y), a.z, s);
    s = fmaf(bf_hi(v.y), a.w, s);
    s = fmaf(bf_lo(v.z), b.x, s);
    s = fmaf(bf_hi(v.z), b.y, s);
    s = fmaf(bf_lo(v.w), b.z, s);
    s = fmaf(bf_hi(v.w), b.w, s);
    return s;
  }
};

// Two e4m3 codes (low byte = first element) to two floats, exactly.
__device__ __forceinline__ float2 e4m3x2(uint32_t two) {
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(two & 0xFFFFu), __NV_E4M3);
  return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}

template <>
struct Unit<PREC_FP8> {
  static constexpr int E = 16;
  __device__ __forceinline__ static void fma4(float *acc, uint32_t w, float x) {
    const float2 a = e4m3x2(w), b = e4m3x2(w >> 16);
    ffma2(acc[0], acc[1], a.x, a.y, x);
    ffma2(acc[2], acc[3], b.x, b.y, x);
  }
  __device__ __forceinline__ static void fma(float *acc, const uint4 &v, float x) {
    fma4(acc + 0, v.x, x);
    fma4(acc + 4, v.y, x);
    fma4(acc + 8, v.z, x);
    fma4(acc + 12, v.w, x);
  }
  // Products with an input x exactly representable in f16 (xh its bits):
  // the decoded f16 weight times x is exact in FP32, and fma.rn.f32.f16
  // rounds the sum once, like the FP32 FMA on the converted weight -- the
  // same sums bit for bit, without converting each weight to FP32.
  __device__ __forceinline__ static void fma4_h(float *acc, uint32_t w, unsigned short xh) {
    const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xFFFFu), __NV_E4M3);
    const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w >> 16), __NV_E4M3);
    asm("{\n\t.reg .f16 x;\n\tmov.b16 x, %8;\n\t"
        "fma.rn.f32.f16 %0, %4, x, %0;\n\tfma.rn.f32.f16 %1, %5, x, %1;\n\t"
        "fma.rn.f32.f16 %2, %6, x, %2;\n\tfma.rn.f32.f16 %3, %7, x, %3;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
        : "h"(lo.x), "h"(lo.y), "h"(hi.x), "h"(hi.y), "h"(xh));
  }
  __device__ __forceinline__ static void fma_h(float *acc, const uint4 &v, unsigned short xh) {
    fma4_h(acc + 0, v.x, xh);
    fma4_h(acc + 4, v.y, xh);
    fma4_h(acc + 8, v.z, xh);
    fma4_h(acc + 12, v.w, xh);
  }
  __device__ __forceinline__ static float dot4(uint32_t w, const float *h, float s) {
    const float2 a = e4m3x2(w), b = e4m3x2(w >> 16);
    const float4 x = *reinterpret_cast<const float4 *>(h);
    s = fmaf(a.x, x.x, s);
    s = fmaf(a.y, x.y, s);
    s = fmaf(b.x, x.z, s);
    s = fmaf(b.y, x.w, s);
    return s;
  }
  __device__ __forceinline__ static float dot(const uint4 &v, const float *h) {
    float s = 0.0f;
    s = dot4(v.x, h, s);
    s = dot4(v.y, h + 4, s);
    s = dot4(v.z, h + 8, s);
    s = dot4(v.w, h + 12, s);
    return s;
  }
};

template <int N>
struct Log2 {
  static constexpr int v = 1 + Log2<N / 2>::v;
};
template <>
struct Log2<1> {
  static constexpr int v = 0;
};

// Finish an input-major layer from each lane's E partial sums:
// out[o] = act(s_o * sum + b_o) for o in [0, H), b_o the sum of nbias bias
// vectors (the paper form's per-sensor input biases), act ReLU or tanh.
// Reduce-scatter over the 32 / UPJ lanes that hold partial sums of the same
// E outputs (xor partners at offsets UPJ, 2 UPJ, ..., 16): at each step a
// lane keeps one half of its live sums, sends the other half to its partner
// and adds the partner's half of what it keeps.  Afterwards every lane
// holds H / 32 finished outputs, so the bias, scale and activation run on
// all 32 lanes.
template <int PREC, int H>
__device__ __forceinline__ void layer_finish(float *acc, const float *__restrict__ bias, int nbias,
                                             const float *__restrict__ scale, float *__restrict__ out,
                                             int lane, int relu) {
  constexpr int E = Unit<PREC>::E;
  constexpr int UPJ = H / E;
  int base = 0;
#pragma unroll
  for (int step = 0; (UPJ << step) < 32; ++step) {
    const int off = UPJ << step;
    constexpr int kE = E;
    const int half = kE >> (step + 1);
    const bool upper = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const float lo = acc[i], hi = acc[i + half];
      const float keep = upper ? hi : lo;
      acc[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, upper ? lo : hi, off);
    }
    if (upper) base += half;
  }
  constexpr int NOUT = H / 32;
  const int o0 = (lane & (UPJ - 1)) * E + base;
#pragma unroll
  for (int i = 0; i < NOUT; ++i) {
    const int o = o0 + i;
    const float s = (PREC == PREC_FP8) ? __ldg(scale + o) : 1.0f;
    float b = __ldg(bias + o);
    for (int k = 1; k < nbias; ++k) b += __ldg(bias + k * H + o);
    const float v = fmaf(acc[i], s, b);
    out[o] = relu ? fmaxf(v, 0.0f) : tanhf(v);
  }
}

// One input-major layer streamed from global memory:
// out[o] = act(s_o * sum_j W[j][o] x[j] + b_o) for o in [0, H), written to
// shared memory.
// SPARSE: stream only the rows of the n_in inputs listed in idx (the
// nonzero entries of x): a row is the H outputs of one input, UPJ whole
// units, so the loads stay 16-byte and contiguous per row.  Skipped inputs
// are exact zeros, whose products add nothing.
template <int PREC, int H, int UNROLL, bool SPARSE>
__device__ __forceinline__ void layer_in_major(const uint4 *__restrict__ w, int n_in,
                                               const float *__restrict__ x,
                                               const float *__restrict__ bias, int nbias,
                                               const float *__restrict__ scale,
                                               float *__restrict__ out, int lane, int relu,
                                               const short *__restrict__ idx, int n_exact = 0) {
  constexpr int E = Unit<PREC>::E;
  constexpr int UPJ = H / E;  // units per input
  constexpr int LG = Log2<UPJ>::v;
  static_assert((1 << LG) == UPJ && UPJ <= 32, "H / E must be a power of two <= 32");
  static_assert(32 * UNROLL * 16 <= kStreamSlack, "a tail batch reads past the layer's end");
  float acc[E];
#pragma unroll
  for (int e = 0; e < E; ++e) acc[e] = 0.0f;
  const int U = n_in * UPJ;
  int u = lane;
  if constexpr (PREC == PREC_FP8 && !SPARSE) {
    // FP8: whole batches whose inputs are all among the first n_exact
    // (exact in f16: the one-hot patch) use the f16-input products
    const int U1 = min(U, (n_exact * UPJ) / (32 * UNROLL) * (32 * UNROLL));
    for (; u < U1; u += 32 * UNROLL) {
      uint4 v[UNROLL];
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) v[k] = ldg_stream(w + u + 32 * k);
#pragma unroll
      for (int k = 0; k < UNROLL; ++k)
        Unit<PREC>::fma_h(acc, v[k], __half_as_ushort(__float2half_rn(x[(u + 32 * k) >> LG])));
    }
  }
  for (; u + 32 * (UNROLL - 1) < U; u += 32 * UNROLL) {
    uint4 v[UNROLL];
    int j[UNROLL];
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) {
      const int uu = u + 32 * k;
      if constexpr (SPARSE) {
        j[k] = idx[uu >> LG];
        v[k] = ldg_stream(w + j[k] * UPJ + (uu & (UPJ - 1)));
      } else {
        j[k] = uu >> LG;
        v[k] = ldg_stream(w + uu);
      }
    }
#pragma unroll
    for (int k = 0; k < UNROLL; ++k) Unit<PREC>::fma(acc, v[k], x[j[k]]);
  }
  if constexpr (PREC == PREC_FP8) {
    // FP8: the last, partial batch (fewer than UNROLL units left for this
    // lane) issues every load before its first product, so the tail costs
    // one memory latency.  Loads run up to 32 * UNROLL units past the
    // layer's end (into the rest of the agent's block, or, after the last
    // block, into the workspace's next kStreamSlack bytes), and the products
    // of those units are skipped, so the products run in the same order as
    // the single-unit loop below.
    if (u < U) {
      uint4 v[UNROLL];
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        if constexpr (SPARSE) {
          const int uu = min(u + 32 * k, U - 1);
          v[k] = ldg_stream(w + idx[uu >> LG] * UPJ + (uu & (UPJ - 1)));
        } else {
          v[k] = ldg_stream(w + u + 32 * k);
        }
      }
#pragma unroll
      for (int k = 0; k < UNROLL; ++k) {
        const int uu = u + 32 * k;
        if (uu < U) Unit<PREC>::fma(acc, v[k], x[SPARSE ? idx[uu >> LG] : uu >> LG]);
      }
    }
  } else {
    for (; u < U; u += 32) {
      if constexpr (SPARSE) {
        const int jj = idx[u >> LG];
        const uint4 v = ldg_stream(w + jj * UPJ + (u & (UPJ - 1)));
        Unit<PREC>::fma(acc, v, x[jj]);
      } else {
        const uint4 v = ldg_stream(w + u);
        Unit<PREC>::fma(acc, v, x[u >> LG]);
      }
    }
  }
  layer_finish<PREC, H>(acc, bias, nbias, scale, out, lane, relu);
}

// Cell one step from (px, py) in direction dir (N E S W) on a torus of side L.
__device__ __forceinline__ int nbr_cell(int px, int py, int dir, int L) {
  int x = px + dir_dx(dir), y = py + dir_dy(dir);
  x += x < 0 ? L : (x >= L ? -L : 0);
  y += y < 0 ? L : (y >= L ? -L : 0);
  return y * L + x;
}

// Observation of one agent (Sec. 3.2 "Sensors"): the k x k x nch patch
// (row, column, channel), then the scalars, into xs.  Lanes 0..3 also read
// the flags of the four neighbouring cells (N E S W) for the move claim:
// *nb_cell = env-local cell, *nb_flags = its cellf byte (lane d: direction d).
__device__ __forceinline__ void gather_obs(const Dev &d, const Layout &L, const Rules &R, int slot,
                                           int env, int pos, int f, float *xs, int lane,
                                           uint32_t kdiv, int *nb_cell, uint32_t *nb_flags) {
  const int k = R.patch_k, RR = k >> 1, kk = k * k;
  const bool rotate = (R.flags & F_ROTATE_OBS) != 0;
  const EnvDesc ed = d.env[env];
  const int side = ed.side;
  const int px = pos % side, py = pos / side;
  const int rt = (f + 1) & 3;
  const uint8_t *cellf = d.cellf + ed.cell_off;
  if (lane < 4) {
    *nb_cell = nbr_cell(px, py, lane, side);
    *nb_flags = cellf[*nb_cell];
  }
  // rows run from far ahead (top) to behind (Around) or to the agent's
  // own row (Front); columns from the agent's left to its right
  const int fw0 = R.view == VIEW_FRONT ? k - 1 : RR;
  const int nch = L.nch;
  const bool terrain = R.rules == RULES_TERRAIN;
  const int rock0 = terrain ? d.rock[ed.cell_off + pos] : 0;
  for (int c = lane; c < kk; c += 32) {
    // c / k by a multiply-high with ceil(2^32 / k): exact for c < 2^10
    const int r = (int)__umulhi((uint32_t)c, kdiv), col = c - r * k;
    int dx, dy;
    if (rotate) {
      const int fw = fw0 - r, ri = col - RR;
      dx = fw * dir_dx(f) + ri * dir_dx(rt);
      dy = fw * dir_dy(f) + ri * dir_dy(rt);
    } else {
      dx = col - RR;
      dy = r - RR;
    }
    // |dx|, |dy| <= k / 2 < side: one correction wraps the torus
    int cx = px + dx, cy = py + dy;
    cx += cx < 0 ? side : (cx >= side ? -side : 0);
    cy += cy < 0 ? side : (cy >= side ? -side : 0);
    const int gc = ed.cell_off + cy * side + cx;
    const uint32_t cf = cellf[cy * side + cx];
    if (R.vision == VISION_RGB) {
      // rendered colours: the occupant's colour trait, else grey wall,
      // else green food (terrain: the cell's biomass, energy and water)
      float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      if (cf & CELL_AGENT) {
        v = d.colour[d.occ[gc]];
      } else if (cf & CELL_WALL) {
        v = make_float4(0.5f, 0.5f, 0.5f, 0.0f);
      } else if (terrain) {
        const float b = (float)d.bio[gc], rr = (float)d.res[gc], w = (float)d.water[gc];
        v = make_float4(b / (b + (float)R.b_bite), rr / (rr + (float)R.e_food), w / (w + (float)R.w_bite), 0.0f);
      } else if (cf & CELL_FOOD) {
        v.y = 1.0f;
      }
      xs[nch * c + 0] = v.x;
      xs[nch * c + 1] = v.y;
      xs[nch * c + 2] = v.z;
      if (terrain) {  // elevation: rock difference d as d / (|d| + 16)
        const float dz = (float)(d.rock[gc] - rock0);
        xs[nch * c + 3] = dz / (fabsf(dz) + 16.0f);
      }
    } else {
      xs[3 * c + 0] = (cf & CELL_FOOD) ? 1.0f : 0.0f;
      xs[3 * c + 1] = (cf & CELL_AGENT) ? 1.0f : 0.0f;
      xs[3 * c + 2] = (cf & CELL_WALL) ? 1.0f : 0.0f;
    }
  }
  if (lane < R.n_scalars) {
    // [e / e_repro, one-hot facing (8-scalar form), zeros]; the paper
    // rules fill the zeros with HP / hp_max, age / (age + age_div) and
    // r / (r + e_food), r the energy lying on the agent's cell
    float v = 0.0f;
    if (lane == 0)
      v = (float)d.energy[slot] / (float)R.e_repro;
    else if (R.n_scalars >= 8 && lane == 1 + f)
      v = 1.0f;
    if (R.rules != RULES_SIMPLE) {
      const int extra = lane - (R.n_scalars >= 8 ? 5 : 1);
      if (extra == 0) {
        v = (float)d.hp[slot] / (float)R.hp_max;
      } else if (extra == 1) {
        const float a = (float)d.age[slot];
        v = a / (a + (float)R.age_div);
      } else if (extra == 2) {
        const float r = (float)d.res[ed.cell_off + pos];
        v = r / (r + (float)R.e_food);
      }
    }
    if (terrain) {  // carried water and biomass; the cell's water and biomass
      if (lane == 8) {
        v = (float)d.a_water[slot] / (float)R.w_cap;
      } else if (lane == 9) {
        v = (float)d.a_bio[slot] / (float)R.b_cap;
      } else if (lane == 10) {
        const float w = (float)d.water[ed.cell_off + pos];
        v = w / (w + (float)R.w_bite);
      } else if (lane == 11) {
        const float b = (float)d.bio[ed.cell_off + pos];
        v = b / (b + (float)R.b_bite);
      }
    }
    xs[nch * kk + lane] = v;
  }
}

// One group of 32 head units (output-major rows of UPJ units): unit u of
// lane u % 32, valid when u < U3; the partial dot products of a row reduce
// over its UPJ lanes, and the row's first lane writes logit a = u / UPJ:
// (W_out h [+ b_out]) * s_a, times exp(-tau) in the paper form.
template <int PREC, int H>
__device__ __forceinline__ void head_group(const uint4 &v, int u, int U3, const float *cur,
                                           const float *__restrict__ out_scale,
                                           const float *__restrict__ hb, int out_bias, int temp,
                                           float tmul, float *ls, int lane) {
  constexpr int E = Unit<PREC>::E;
  constexpr int UPJ = H / E;
  constexpr int LG = Log2<UPJ>::v;
  float part = 0.0f;
  if (u < U3) part = Unit<PREC>::dot(v, cur + (u & (UPJ - 1)) * E);
#pragma unroll
  for (int off = 1; off < UPJ; off <<= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, off);
  if (u < U3 && (lane & (UPJ - 1)) == 0) {
    const int a = u >> LG;
    const float s = (PREC == PREC_FP8) ? __ldg(out_scale + a) : 1.0f;
    const float val = out_bias ? fmaf(part, s, __ldg(hb + a)) : part * s;
    ls[a] = temp ? val * tmul : val;
  }
}

// Sample the action (Sec. 3.3: argmax_a (logit_a + Gumbel_a), ties to the
// lowest a; GREEDY: argmax of the logits), store the logits and the
// action, and, with apply_moves, the fused part of A6: facing and turns,
// and the move claim on a cell that is neither a wall nor occupied now, at
// the start of the step (no cell changes while the policy phase runs).
// Lane A draws the agent's CLAIM_MOVE number in the same pass as lanes
// 0..A-1 draw their Gumbel noise; lanes 0..3 hold the neighbouring cells
// and their flags (gather_obs).  Counts into the warp's counters: lane a <
// 16 action a, lane 16 moves blocked by a wall or an agent.
__device__ __forceinline__ void sample_and_claim(const Dev &d, const Rules &R, int A, int slot, int env,
                                                 int pos, int f, const float *ls, int lane, uint32_t t,
                                                 bool greedy, int apply_moves, int nb_cell,
                                                 uint32_t nb_flags, int &cnt) {
  float score = -INFINITY;
  int best = lane;
  uint32_t claim_r = 0;
  if (lane <= A) {
    const EnvDesc ed = d.env[env];
    const bool claimer = lane == A;
    float lg = 0.0f;
    if (!claimer) {
      lg = ls[lane];
      d.logits[(int64_t)slot * A + lane] = lg;
      score = lg;
    }
    if (claimer ? apply_moves != 0 : !greedy) {
      const U4 r = philox(t, (uint32_t)(slot - ed.slot_off), claimer ? 0u : (uint32_t)(lane >> 2), 0u,
                          ed.seed, claimer ? S_CLAIM_MOVE : S_SAMPLE);
      if (claimer) {
        claim_r = r.x;
      } else {
        const float u = uniform01(word_of(r, lane & 3));
        score = lg + (-logf(-logf(u)));
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float os = __shfl_xor_sync(0xFFFFFFFFu, score, off);
    const int oa = __shfl_xor_sync(0xFFFFFFFFu, best, off);
    if (os > score || (os == score && oa < best)) {
      score = os;
      best = oa;
    }
  }
  if (apply_moves) {
    int nf = f;
    bool move = false;
    if (R.rules != RULES_SIMPLE) {
      // rotate clockwise / counter-clockwise, or one cell forward
      if (best == PA_CW) nf = (f + 1) & 3;
      else if (best == PA_CCW) nf = (f + 3) & 3;
      move = best == PA_FORWARD;
    } else if (best >= ACT_N && best <= ACT_W) {
      nf = (best == ACT_N) ? 0 : (best == ACT_S) ? 2 : (best == ACT_E) ? 1 : 3;
      move = true;
    } else if (best == ACT_LEFT) {
      nf = (f + 3) & 3;
    } else if (best == ACT_RIGHT) {
      nf = (f + 1) & 3;
    }
    const int c = __shfl_sync(0xFFFFFFFFu, nb_cell, nf);
    const uint32_t cf = __shfl_sync(0xFFFFFFFFu, nb_flags, nf);
    const uint32_t draw = __shfl_sync(0xFFFFFFFFu, claim_r, A);
    const int blk = (move && (cf & (CELL_WALL | CELL_AGENT))) ? 1 : 0;
    if (lane == 0) {
      int tc = -1;
      if (move && !blk) {
        const EnvDesc ed = d.env[env];
        const int local = slot - ed.slot_off;
        atomicMax(&d.claim_move[ed.cell_off + c], claim_key(draw, local));
        if (R.flags & F_CANCEL_ALL) atomicAdd(&d.cnt_move[ed.cell_off + c], 1u);
        tc = c;
      }
      d.facing[slot] = (uint8_t)nf;
      d.tgt[slot] = tc;
    }
    if (lane == best) ++cnt;
    if (lane == 16 && blk) ++cnt;
  }
  if (lane == 0) d.act[slot] = (uint8_t)best;
}

// The weight stream is latency-bound per warp: the register budget is capped
// so that MINB CTAs (MINB * WARPS warps) stay resident per SM -- about 40
// warps at 48 registers, or 32 warps at 64 registers for the FP8 form, whose
// 16 accumulators per lane need the room.
template <int PREC, int H, int WARPS, int UNROLL, int MINB, bool SPARSE>
__global__ void __launch_bounds__(WARPS * 32, MINB)
    k_policy(Dev d, Layout L, Rules R, int xs_floats, int apply_moves) {
  constexpr int E = Unit<PREC>::E;
  constexpr int UPJ = H / E;
  extern __shared__ __align__(16) float smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // per warp: observation (then a hidden activation), hidden activation,
  // logits, and for SPARSE the list of the nonzero inputs (shorts)
  float *xs = smem + warp * policy_warp_floats(xs_floats, H, SPARSE);
  float *hs = xs + xs_floats;
  float *ls = hs + H;

  const int n_alive = d.counters[CNT_N_ALIVE];
  const uint32_t t = (uint32_t)d.step[0];
  // the step's agent count, for the byte count of timed launches
  if (apply_moves && blockIdx.x == 0 && threadIdx.x == 0) d.alive_at_step[t & (kAliveRing - 1)] = n_alive;
  const int k = R.patch_k;
  // ceil(2^32 / k) for odd k (k = 0: no patch, the gather loop is empty)
  const uint32_t kdiv = k > 0 ? 0xFFFFFFFFu / (uint32_t)k + 1u : 0u;
  const bool greedy = (R.flags & F_GREEDY) != 0;

  // Per-warp counters, flushed when the environment changes: lane a < 16
  // counts action a, lane 16 counts moves blocked by a wall or an agent.
  int cnt = 0, e_cur = -1;
  auto flush = [&]() {
    if (e_cur >= 0 && cnt && lane <= 16)
      atomicAdd((unsigned long long *)&d.stats_step[e_cur * N_ST + (lane < 16 ? ST_ACT0 + lane : ST_MOVE_BLOCKED)],
                (unsigned long long)cnt);
    cnt = 0;
  };

  // Balanced rounds (BF16, FP32): the launch needs R = ceil(n_alive / G)
  // rounds of its G resident warps; only the first ceil(n_alive / R) warps
  // take agents, so every round keeps the same number of warps streaming
  // instead of the last one running on a fraction of them.  (CTAs are
  // spread over the SMs in turn, so the idle warps are spread too.)  Each
  // agent is still one warp's, computed the same way.  The FP8 form, whose
  // warps spend more of their time issuing, loses more from the fewer warps
  // in every round than it gains in the last one, and keeps all G.
  const int G = gridDim.x * WARPS;
  const int rounds = (n_alive + G - 1) / G;
  const int G_eff = (PREC != PREC_FP8 && rounds > 0) ? (n_alive + rounds - 1) / rounds : G;
  const int w0 = blockIdx.x * WARPS + warp;
  // At the start of the launch every warp gathers an observation with no
  // weights in flight: the first 4 KB of each warp's first agent's weights
  // are requested into L2 before that gather.
  if (lane == 0 && w0 < G_eff && w0 < n_alive)
    prefetch_l2(d.wq + (int64_t)d.alive_list[w0] * L.stride, (uint32_t)min((int64_t)4096, (int64_t)L.off_w2));
  // The next agent's slot is read one agent ahead, and its environment,
  // cell and facing while the current agent's head is computed, so a new
  // agent starts with its observation gather.  (A slot's facing is written
  // only by the warp that computes it, in its own iteration.)
  int i = w0 < G_eff ? w0 : n_alive;
  int slot_n = 0, env_n = 0, pos_n = 0, f_n = 0;
  if (i < n_alive) {
    slot_n = d.alive_list[i];
    env_n = d.env_of[slot_n];
    pos_n = d.pos[slot_n];
    f_n = d.facing[slot_n];
  }
  for (; i < n_alive; i += G_eff) {
    const int slot = slot_n, env = env_n, pos = pos_n, f = f_n;
    const bool more = i + G_eff < n_alive;
    if (more) slot_n = d.alive_list[i + G_eff];
    if (env != e_cur) {
      flush();
      e_cur = env;
    }
    int nb_cell = 0;
    uint32_t nb_flags = 0;
    gather_obs(d, L, R, slot, env, pos, f, xs, lane, kdiv, &nb_cell, &nb_flags);
    __syncwarp();

    const uint8_t *blk = d.wq + (int64_t)slot * L.stride;
    const uint4 *wb = reinterpret_cast<const uint4 *>(blk);
    const float *bias = reinterpret_cast<const float *>(blk + L.off_bias);
    const float *scale = reinterpret_cast<const float *>(blk + L.off_scale);

    // -- input layer: act(sum over sensors of (W_s x_s + b_s)) -> hs
    if constexpr (SPARSE) {
      // list the nonzero inputs in ascending order (a warp ballot per 32)
      short *idx = reinterpret_cast<short *>(ls + 16);
      int n_nz = 0;
      for (int base = 0; base < L.D; base += 32) {
        const int j = base + lane;
        const bool nz = j < L.D && xs[j] != 0.0f;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, nz);
        if (nz) idx[n_nz + __popc(m & ((1u << lane) - 1u))] = (short)j;
        n_nz += __popc(m);
      }
      __syncwarp();
      layer_in_major<PREC, H, UNROLL, true>(wb + L.off_w1 / 16, n_nz, xs, bias, L.ns, scale, hs,
                                            lane, L.relu, idx);
    } else {
      // one-hot vision: the patch inputs are 0 or 1, exact in f16
      layer_in_major<PREC, H, UNROLL, false>(wb + L.off_w1 / 16, L.D, xs, bias, L.ns, scale, hs,
                                             lane, L.relu, nullptr,
                                             R.vision == VISION_CHANNELS ? L.patch : 0);
    }
    __syncwarp();
    // -- hidden layers: h = act(W_l h + b_l), alternating between hs and xs
    float *cur = hs, *nxt = xs;
    for (int l = 0; l < L.L; ++l) {
      layer_in_major<PREC, H, UNROLL, false>(wb + (L.off_w2 + l * H * H * L.es) / 16, H, cur,
                                             bias + L.ns * H + l * H, 1, scale + H + l * H, nxt,
                                             lane, L.relu, nullptr);
      __syncwarp();
      float *tmp = cur;
      cur = nxt;
      nxt = tmp;
    }

    if (more) {
      env_n = d.env_of[slot_n];
      pos_n = d.pos[slot_n];
      f_n = d.facing[slot_n];
    }
    // -- head: logits = (W_out h [+ b_out]) / exp(tau) (output-major rows of
    //    H / E units; the temperature only in the paper form)
    const uint4 *w3 = wb + L.off_w3 / 16;
    const int U3 = L.A * UPJ;
    const float *hb = bias + L.ns * H + L.L * H;  // head bias, then tau
    const float tmul = L.temp ? expf(-__ldg(hb + (L.out_bias ? L.A : 0))) : 1.0f;
    // the head's groups of 32 units, up to kHeadBatch of them requested
    // before the first one is reduced
    constexpr int kHeadBatch = 4;
    for (int base = 0; base < U3; base += 32 * kHeadBatch) {
      uint4 hv[kHeadBatch];
#pragma unroll
      for (int g = 0; g < kHeadBatch; ++g) {
        const int u = base + 32 * g + lane;
        hv[g] = u < U3 ? ldg_stream(w3 + u) : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int g = 0; g < kHeadBatch; ++g)
        if (base + 32 * g < U3)
          head_group<PREC, H>(hv[g], base + 32 * g + lane, U3, cur, scale + H + L.L * H, hb, L.out_bias,
                              L.temp, tmul, ls, lane);
    }
    __syncwarp();

    sample_and_claim(d, R, L.A, slot, env, pos, f, ls, lane, t, greedy, apply_moves, nb_cell, nb_flags, cnt);
    __syncwarp();
  }
  flush();
}

// ---------------------------------------------------------------------------
// Variant k (1-based) of one precision and hidden width.  Variants 7 and 8
// are the input-sparse forms of 3 and 6 (they stream only the W_in rows of
// nonzero inputs); the autotuner keeps the two families apart.  Variants 9
// and 10 sit between the 48- and 64-register ones: 56 registers, 36 warps
// per SM.
// ---------------------------------------------------------------------------
template <int PREC, int H>
PolicyFn policy_pick_variant(int variant) {
  switch (variant) {
    case 1: return k_policy<PREC, H, 4, 8, 10, false>;
    case 2: return k_policy<PREC, H, 8, 8, 5, false>;
    case 3: return k_policy<PREC, H, 8, 4, 5, false>;
    case 4: return k_policy<PREC, H, 16, 4, 2, false>;
    case 5: return k_policy<PREC, H, 8, 4, 4, false>;
    case 6: return k_policy<PREC, H, 4, 8, 8, false>;
    case 7: return k_policy<PREC, H, 8, 4, 5, true>;
    case 8: return k_policy<PREC, H, 4, 8, 8, true>;
    case 9: return k_policy<PREC, H, 4, 8, 9, false>;
    case 10: return k_policy<PREC, H, 4, 4, 9, false>;
    default: return nullptr;
  }
}

template <int PREC>
PolicyFn policy_pick_width(int H, int variant) {
  if (H == 32) return policy_pick_variant<PREC, 32>(variant);
  if (H == 64) return policy_pick_variant<PREC, 64>(variant);
  if (H == 128) return policy_pick_variant<PREC, 128>(variant);
  return nullptr;
}

}  // namespace eco
