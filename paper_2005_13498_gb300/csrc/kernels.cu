// Batched Hubbard-apply and Lanczos kernels for sm_103a.
//
// Psi of a sector is a dim_up x dim_dn row-major matrix.  H acts as
//   W[u,d] = sum_{(u',g,s) in C_up(u)} s c_g Psi[u',d]      (T_up: across rows)
//          + sum_{(d',g,s) in C_dn(d)} s c_g Psi[u,d']      (T_dn: within a row)
//          + (U popcount(up[u] & dn[d]) + eps_up[u] + eps_dn[d]) Psi[u,d]
// (Eq. (1) with the Peierls phases of Eq. (3); c_g the per-step coefficient of
// bond class g/2 in orientation g%2).  One CTA processes a block of rows u:
// the rows Psi[u,:] are staged in shared memory for T_dn, the T_up gathers
// read whole rows Psi[u',:] with coalesced loads along d, and the signed
// values of one bond group are summed before a single complex multiply by
// c_g.  The column index d is a position in the down-spin table's basis
// order (ascending words, or the hop order the propagation uses).
//
// The Lanczos recursion (Algorithm 6) is split into two passes per step j:
//   apply :  w = s_j H x_j - beta_{j-1} s_{j-1} x_{j-1},  alpha_j = Re<v_j, w>
//   update:  x_{j+1} = w - alpha_j s_j x_j,  beta_j = |x_{j+1}|,
//            s_{j+1} = 1 / beta_j   (normalisation is applied lazily)
// Reductions are deterministic: per-block partial sums in float64, then the
// last block of each vector sums the partials in block order.
#include "kernels.cuh"

#include <cstdio>

namespace ed {

// ---------------------------------------------------------------- utilities
template <typename R> struct C2T;
template <> struct C2T<float> { using T = float2; };
template <> struct C2T<double> { using T = double2; };

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

// Two independent round-to-nearest FP32 FMAs in one packed instruction
// (fma.rn.f32x2, sm_100 and later): (a.x b.x + c.x, a.y b.y + c.y), the same
// values as two scalar FMAs.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long ra, rb, rc, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rc) : "f"(c.x), "f"(c.y));
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
// s += g v (complex s, v; real g)
template <typename C, typename R>
__device__ __forceinline__ void cax(C& s, R g, const C& v) {
  if constexpr (sizeof(R) == 4) {
    s = ffma2(make_float2(g, g), v, s);
  } else {
    s.x += g * v.x;
    s.y += g * v.y;
  }
}
// acc += c s (complex), each component a chain of two fused multiply-adds
// into acc: no product is rounded on its own (two FMAs per component, where
// acc + (a b - c d) takes a multiply, an FMA and an add)
template <typename C>
__device__ __forceinline__ void cmac(C& acc, const C c, const C s) {
  if constexpr (sizeof(C) == 8) {
    acc = ffma2(make_float2(c.x, c.x), s, acc);
    acc = ffma2(make_float2(-c.y, c.y), make_float2(s.y, s.x), acc);
  } else {
    acc.x = __fma_rn(-c.y, s.y, __fma_rn(c.x, s.x, acc.x));
    acc.y = __fma_rn(c.y, s.x, __fma_rn(c.x, s.y, acc.y));
  }
}
// the same for the two complex64 values of a 16-byte word
__device__ __forceinline__ void cmac4(float4& acc, const float2 c, const float4 s) {
  float2 a = make_float2(acc.x, acc.y), b = make_float2(acc.z, acc.w);
  cmac(a, c, make_float2(s.x, s.y));
  cmac(b, c, make_float2(s.z, s.w));
  acc = make_float4(a.x, a.y, b.x, b.y);
}

template <typename R> __device__ __forceinline__ typename C2T<R>::T
load_coef(const void* p, int idx) {
  return reinterpret_cast<const typename C2T<R>::T*>(p)[idx];
}

// Block reduction of K doubles; the result is valid in thread 0.
template <int K>
__device__ __forceinline__ void block_reduce(double (&v)[K], double* red) {
  const unsigned full = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < K; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(full, v[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[wid * K + k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      v[k] = lane < nw ? red[lane * K + k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(full, v[k], o);
    }
  }
}

// Write this block's partials; the last block of [b0, b1) sums all partials
// in block order.  Returns true in every thread of the last block; the totals
// are valid in thread 0.
template <int K>
__device__ __forceinline__ bool reduce_last_block(double (&v)[K], int blk, int b0,
                                                  int b1, double* partials,
                                                  unsigned* counter,
                                                  double* red, int* flag) {
  block_reduce<K>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[(size_t)blk * K + k] = v[k];
    __threadfence();
    unsigned ticket = atomicAdd(counter, 1u);
    *flag = (ticket == (unsigned)(b1 - b0 - 1));
  }
  __syncthreads();
  if (!*flag) return false;
  __threadfence();
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] += __ldcg(&partials[(size_t)b * K + k]);
  block_reduce<K>(acc, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = acc[k];
    *counter = 0u;
  }
  return true;
}

// Whether the Lanczos passes of step j are skipped: after a breakdown, or
// once the adaptive check of a step <= j - 2 has converged.  The check of
// step j - 1 runs concurrently with pass j (its result must not change
// pass j's decision halfway through the grid: conv_m = j - 1 fails the test),
// and the pass j + 1 kernels start after it has finished.
__device__ __forceinline__ bool lanczos_done(const LanczosState* st, int j) {
  const int c = *(volatile const int*)&st->conv_m;
  return st->stopped || (c > 0 && c <= j - 2);
}

__device__ __forceinline__ const void* xptr(const VecDev& vd, int j, size_t esz) {
  // x_1 is the state, x_j (j >= 2) is V slot j-2
  return j == 1 ? vd.x1
                : static_cast<const char*>(vd.V) + (size_t)(j - 2) * vd.D * esz;
}

// ------------------------------------------------------------------- apply
// j >= 1: Lanczos pass j; j == 0: plain apply (coefs row 0, x1 -> w);
// j == -1: energy of x1 with coefs_obs[step].
// (The apply kernel and its phases are described at k_apply below.)

// ---- TMA pipeline for the T_up row segments (TMA apply configurations).
// A producer warp copies the source-row chunk of every T_up entry into a ring
// of shared-memory slots (the configuration's stage count) with
// cp.async.bulk; "full" mbarriers carry the byte count, "empty" mbarriers
// collect one arrival per consumer warp.  Every wait is bounded: after
// BatchArgs::wait_limit failed polls the thread records ED_ERR_TIMEOUT in the
// vector's status and a block-wide flag, and all later waits of the block
// give up at once.
constexpr int kStatusTimeout = 4;    // ED_ERR_TIMEOUT

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase of the given parity; false on timeout or when
// another thread of the block has already timed out (err set).
// The flag is tested before every poll: once a wait of the block has given
// up, a later slot's barrier may still be in the phase of a copy that was
// never issued, and a poll for the other parity would report that phase as
// complete (the parity names the previous phase).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* err,
                                          uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (*err) return false;
    if (mbar_try_wait(bar, parity)) return true;
  }
  *err = 1;
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple
// of 16), completing bytes on the mbarrier.
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                             uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Column pair (2p, 2p+1) of a row: one 16-byte access for aligned complex64
// rows (VEC), else two element accesses with the second column checked.
// STREAM: data read or written once in this pass (the previous Krylov vector,
// the output w): evict-first cache hints, so that the vector whose rows are
// gathered stays in L2.
template <typename C, bool VEC, bool STREAM = false>
__device__ __forceinline__ void load_pair(const C* row, int p, int dim, C& v0, C& v1) {
  if constexpr (VEC) {
    const float4* a = reinterpret_cast<const float4*>(row) + p;
    const float4 f = STREAM ? __ldcs(a) : *a;
    v0.x = f.x; v0.y = f.y; v1.x = f.z; v1.y = f.w;
  } else {
    const int d = 2 * p;
    v0 = STREAM ? __ldcs(row + d) : row[d];
    if (d + 1 < dim) v1 = STREAM ? __ldcs(row + d + 1) : row[d + 1]; else v1 = czero<C>();
  }
}
template <typename C, bool VEC, bool STREAM = false>
__device__ __forceinline__ void store_pair(C* row, int p, int dim, C v0, C v1) {
  if constexpr (VEC) {
    float4* a = reinterpret_cast<float4*>(row) + p;
    const float4 f = make_float4(v0.x, v0.y, v1.x, v1.y);
    if (STREAM) __stcs(a, f); else *a = f;
  } else {
    const int d = 2 * p;
    if (STREAM) __stcs(row + d, v0); else row[d] = v0;
    if (d + 1 < dim) { if (STREAM) __stcs(row + d + 1, v1); else row[d + 1] = v1; }
  }
}

template <typename R>
__device__ __forceinline__ R sign_of(uint32_t ent) {
  // +1 or -1 from bit 31
  if constexpr (sizeof(R) == 4) return __int_as_float((int)((ent & 0x80000000u) | 0x3f800000u));
  else return (ent & 0x80000000u) ? -1.0 : 1.0;
}

// Shared-memory tile of NR rows, stored column by column.  When the NR values
// of a column fill two 16-byte chunks (complex64 x 4 rows, complex128 x 2
// rows) the two chunks of column d are swapped for d mod 8 >= 4, so that the
// chunk a lane reads for a random column lands in any of the eight 16-byte
// bank groups (bank conflicts of random column gathers drop by about half).
template <typename C, int NR>
struct TileIO {
  static constexpr int kBytes = NR * (int)sizeof(C);
  __device__ static __forceinline__ void load(const C* tile, int d, C (&v)[NR]) {
    if constexpr (kBytes == 32) {
      const float4* t = reinterpret_cast<const float4*>(tile);
      const int sw = (d >> 2) & 1;
      const float4 a = t[2 * d + sw], b = t[2 * d + (sw ^ 1)];
      if constexpr (sizeof(C) == 8) {
        v[0].x = a.x; v[0].y = a.y; v[1].x = a.z; v[1].y = a.w;
        v[2].x = b.x; v[2].y = b.y; v[3].x = b.z; v[3].y = b.w;
      } else {
        v[0] = *reinterpret_cast<const C*>(&a);
        v[1] = *reinterpret_cast<const C*>(&b);
      }
    } else if constexpr (kBytes == 16) {
      const float4 a = reinterpret_cast<const float4*>(tile)[d];
      v[0] = *reinterpret_cast<const C*>(&a);
      if constexpr (NR == 2) v[1] = *(reinterpret_cast<const C*>(&a) + 1);
    } else {
#pragma unroll
      for (int r = 0; r < NR; ++r) v[r] = tile[(size_t)d * NR + r];
    }
  }
  // load by a table entry: the byte offset of the column (of its first
  // chunk, tile_offset, for 32-byte columns) from the ELL copy of this
  // column width (ell_for)
  __device__ static __forceinline__ void load_ent(const C* tile, uint32_t ent, C (&v)[NR]) {
    const uint32_t off = ent & 0x7FFFFFFFu;
    if constexpr (kBytes == 32) {
      const char* base = reinterpret_cast<const char*>(tile);
      const float4 a = *reinterpret_cast<const float4*>(base + off);
      const float4 b = *reinterpret_cast<const float4*>(base + (off ^ 16u));
      if constexpr (sizeof(C) == 8) {
        v[0].x = a.x; v[0].y = a.y; v[1].x = a.z; v[1].y = a.w;
        v[2].x = b.x; v[2].y = b.y; v[3].x = b.z; v[3].y = b.w;
      } else {
        v[0].x = __longlong_as_double(((long long)__float_as_int(a.y) << 32) | (unsigned)__float_as_int(a.x));
        v[0].y = __longlong_as_double(((long long)__float_as_int(a.w) << 32) | (unsigned)__float_as_int(a.z));
        v[1].x = __longlong_as_double(((long long)__float_as_int(b.y) << 32) | (unsigned)__float_as_int(b.x));
        v[1].y = __longlong_as_double(((long long)__float_as_int(b.w) << 32) | (unsigned)__float_as_int(b.z));
      }
    } else if constexpr (kBytes == 16) {
      const float4 a = *reinterpret_cast<const float4*>(reinterpret_cast<const char*>(tile) + off);
      if constexpr (sizeof(C) == 8) {
        v[0].x = a.x; v[0].y = a.y; v[1].x = a.z; v[1].y = a.w;
      } else {
        v[0].x = __longlong_as_double(((long long)__float_as_int(a.y) << 32) | (unsigned)__float_as_int(a.x));
        v[0].y = __longlong_as_double(((long long)__float_as_int(a.w) << 32) | (unsigned)__float_as_int(a.z));
      }
    } else if constexpr (kBytes == 8) {
      v[0] = *reinterpret_cast<const C*>(reinterpret_cast<const char*>(tile) + off);
    } else {
      load(tile, (int)(off >> 5), v);
    }
  }
  // load by a byte offset: of the column (of its first chunk for 32-byte
  // columns, whose second chunk is at offset ^ 16)
  __device__ static __forceinline__ void load_off(const C* tile, uint32_t off, C (&v)[NR]) {
    load_ent(tile, off, v);
  }
  // packed ELL word of one lane and slot: bits 0-14 the column unit of the
  // lane's first column's entry, bit 15 the sign of the second, bits 16-30
  // the unit of the second, bit 31 the sign of the first; a unit is 8 bytes
  // for 8-byte columns and 16 bytes otherwise (only 8-, 16- and 32-byte
  // columns occur in the configuration table)
  static_assert(kBytes == 8 || kBytes == 16 || kBytes == 32, "packed ELL column widths");
  static constexpr int kUnitShift = kBytes == 8 ? 3 : 4;
  template <typename R>
  __device__ static __forceinline__ void unpack(uint32_t e, uint32_t& off0, uint32_t& off1,
                                                R& g0, R& g1) {
    off0 = (e & 0x7FFFu) << kUnitShift;
    off1 = ((e >> 16) & 0x7FFFu) << kUnitShift;
    g0 = sign_of<R>(e);
    g1 = sign_of<R>(e << 16);
  }
  __device__ static __forceinline__ const uint32_t* ellp_for(const uint32_t* p32,
                                                             const uint32_t* prank) {
    if constexpr (kBytes == 32) return p32;
    else return prank;
  }
  // the ELL copy whose entries hold byte offsets for this column width
  __device__ static __forceinline__ const uint32_t* ell_for(const uint32_t* ell32,
                                                            const uint32_t* ell16,
                                                            const uint32_t* ell8) {
    if constexpr (kBytes == 16) return ell16;
    else if constexpr (kBytes == 8) return ell8;
    else return ell32;
  }
  __device__ static __forceinline__ void store(C* tile, int d, const C (&v)[NR]) {
    if constexpr (kBytes == 32) {
      float4* t = reinterpret_cast<float4*>(tile);
      const int sw = (d >> 2) & 1;
      float4 a, b;
      if constexpr (sizeof(C) == 8) {
        a = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        b = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
      } else {
        a = *reinterpret_cast<const float4*>(&v[0]);
        b = *reinterpret_cast<const float4*>(&v[1]);
      }
      t[2 * d + sw] = a;
      t[2 * d + (sw ^ 1)] = b;
    } else if constexpr (kBytes == 16) {
      float4 a;
      *reinterpret_cast<C*>(&a) = v[0];
      if constexpr (NR == 2) *(reinterpret_cast<C*>(&a) + 1) = v[1];
      reinterpret_cast<float4*>(tile)[d] = a;
    } else {
#pragma unroll
      for (int r = 0; r < NR; ++r) tile[(size_t)d * NR + r] = v[r];
    }
  }
};

// T_up gathers of one chunk of the apply (k_apply): for each of the CTA's
// rows u the entry list of u (uniform over the block) is walked four entries
// at a time, each a coalesced load of the thread's column pairs of the
// source row per column-pair group k < KA, all loads of a batch in flight
// before they are used; the last 1-3 entries of a list form a batch of their
// own (complex64: one batch of three guarded by the count, which keeps the
// configurations free of spills; complex128: a batch of each size), so no
// load serves a padding entry (the lists are stored padded to 4 entries,
// which keeps their 16-byte metadata loads aligned).  KA counts the groups of this chunk that hold valid pairs; in
// the last of them the pair index is clamped to the last pair of the row
// (those sums are never stored).
//  * complex64: no group sums.  Each entry reads its signed coefficient
//    s c_g from the CTA's table coefQ[cs] = (s Re c, s Re c, s Im c, s Im c)
//    (cs = 1 + 2 g + [s < 0]), one broadcast load, and accumulates
//    a += (Re, Re) v, b += (Im, Im) v with two packed FMAs and no operand
//    swaps; the row ends with acc += (a.x - b.y, a.y + b.x).
//  * complex128 (FP64-pipe bound): signed sums per bond group, multiplied
//    by c_g once per group.
template <int NB, int KA, bool VEC>
__device__ __forceinline__ void tup_batch_c64(const float2* xrow, const int (&pk)[KA],
                                              const float4* coefQ, int dim_dn,
                                              const uint32_t (&css)[4], const uint32_t (&rows)[4],
                                              float2 (&sa)[2 * KA], float2 (&sb)[2 * KA],
                                              int nb = NB) {
  float2 v[NB][2 * KA];   // entries qq >= nb (uniform over the block) are not read
#pragma unroll
  for (int qq = 0; qq < NB; ++qq) {
    if (qq >= nb) {
#pragma unroll
      for (int k = 0; k < 2 * KA; ++k) v[qq][k] = make_float2(0.f, 0.f);
      continue;
    }
    const float2* src = xrow + rows[qq];
#pragma unroll
    for (int k = 0; k < KA; ++k) {
      if constexpr (VEC) {
        const float4 f = __ldcg(reinterpret_cast<const float4*>(src) + pk[k]);
        v[qq][2 * k] = make_float2(f.x, f.y);
        v[qq][2 * k + 1] = make_float2(f.z, f.w);
      } else {
        load_pair<float2, false>(src, pk[k], dim_dn, v[qq][2 * k], v[qq][2 * k + 1]);
      }
    }
  }
#pragma unroll
  for (int qq = 0; qq < NB; ++qq) {
    if (qq >= nb) continue;
    const float4 q = coefQ[css[qq]];
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) {
      sa[k] = ffma2(make_float2(q.x, q.y), v[qq][k], sa[k]);
      sb[k] = ffma2(make_float2(q.z, q.w), v[qq][k], sb[k]);
    }
  }
}

template <int NR, int PP, int KA, bool VEC, int NT>
__device__ __forceinline__ void tup_chunk_c64(const SectorDev& sd,
                                              const float2* const (&xr)[NR],
                                              const float4* coefQ, const int (&urow)[NR],
                                              int nrows, int pc,
                                              int npairs, int dim_dn, float2 (&acc)[NR][2 * PP]) {
  constexpr int T = NT;
  int pk[KA];
#pragma unroll
  for (int k = 0; k < KA; ++k) pk[k] = min(pc + (int)threadIdx.x + k * T, npairs - 1);
  const uint4* cs4p = reinterpret_cast<const uint4*>(sd.up_pad_cs);
  const uint4* row4p = reinterpret_cast<const uint4*>(sd.up_pad_row);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r >= nrows) continue;   // uniform over the block
    const int u = urow[r];
    const int e0 = __ldg(sd.up_pad_off + u);
    const int e1 = e0 + (__ldg(sd.up_off + u + 1) - __ldg(sd.up_off + u));   // real entries
    if (e0 >= e1) continue;
    float2 sa[2 * KA], sb[2 * KA];
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) { sa[k] = make_float2(0.f, 0.f); sb[k] = sa[k]; }
    uint4 ncs = __ldg(cs4p + (e0 >> 2)), nrow = __ldg(row4p + (e0 >> 2));
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
      const uint32_t css[4] = {ncs.x, ncs.y, ncs.z, ncs.w};
      const uint32_t rows[4] = {nrow.x, nrow.y, nrow.z, nrow.w};
      if (e + 4 < e1) {   // the next batch's entries load under this batch's rows
        ncs = __ldg(cs4p + ((e + 4) >> 2));
        nrow = __ldg(row4p + ((e + 4) >> 2));
      }
      tup_batch_c64<4, KA, VEC>(xr[r], pk, coefQ, dim_dn, css, rows, sa, sb);
    }
    if (e < e1) {   // the last 1-3 entries (uniform over the block)
      const uint32_t css[4] = {ncs.x, ncs.y, ncs.z, ncs.w};
      const uint32_t rows[4] = {nrow.x, nrow.y, nrow.z, nrow.w};
      const int nb = e1 - e;
      tup_batch_c64<3, KA, VEC>(xr[r], pk, coefQ, dim_dn, css, rows, sa, sb, nb);
    }
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) {
      acc[r][k].x += sa[k].x - sb[k].y;
      acc[r][k].y += sa[k].y + sb[k].x;
    }
  }
}

// complex128: row r gathers from xr[r] (one vector, or one per row in
// multi-vector blocks); the signed values of a bond group are summed and
// multiplied by c_g when the group changes
template <int NB, int KA, int PP>
__device__ __forceinline__ void tup_batch_c128(const double2* xrow, const int (&pk)[KA],
                                               int dim_dn, const uint32_t (&ents)[4],
                                               const uint32_t (&rows)[4], const double2* coefS,
                                               double2 (&sum)[2 * KA], uint32_t& gcur,
                                               double2 (&accr)[2 * PP]) {
  using C = double2;
  C v[NB][2 * KA];
#pragma unroll
  for (int qq = 0; qq < NB; ++qq)
#pragma unroll
    for (int k = 0; k < KA; ++k)
      load_pair<C, false>(xrow + rows[qq], pk[k], dim_dn, v[qq][2 * k], v[qq][2 * k + 1]);
#pragma unroll
  for (int qq = 0; qq < NB; ++qq) {
    const uint32_t g = (ents[qq] >> kEntGroupShift) & 0xFFu;
    if (g != gcur) {                              // uniform over the block
      const C c = coefS[gcur];
#pragma unroll
      for (int k = 0; k < 2 * KA; ++k) {
        cmac(accr[k], c, sum[k]);
        sum[k] = czero<C>();
      }
      gcur = g;
    }
    const double sg = sign_of<double>(ents[qq]);
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) cax(sum[k], sg, v[qq][k]);
  }
}

template <int NR, int PP, int KA, int NT>
__device__ __forceinline__ void tup_chunk_c128(const SectorDev& sd,
                                               const double2* const (&xr)[NR],
                                               const double2* coefS, const int (&urow)[NR],
                                               int nrows, int pc,
                                               int npairs, int dim_dn,
                                               double2 (&acc)[NR][2 * PP]) {
  using C = double2;
  constexpr int T = NT;
  int pk[KA];
#pragma unroll
  for (int k = 0; k < KA; ++k) pk[k] = min(pc + (int)threadIdx.x + k * T, npairs - 1);
  const uint4* ent4p = reinterpret_cast<const uint4*>(sd.up_pad_ent);
  const uint4* row4p = reinterpret_cast<const uint4*>(sd.up_pad_row);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if (r >= nrows) continue;   // uniform over the block
    const int u = urow[r];
    const int e0 = __ldg(sd.up_pad_off + u);
    const int e1 = e0 + (__ldg(sd.up_off + u + 1) - __ldg(sd.up_off + u));   // real entries
    if (e0 >= e1) continue;
    C sum[2 * KA];
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) sum[k] = czero<C>();
    uint4 nent = __ldg(ent4p + (e0 >> 2)), nrow = __ldg(row4p + (e0 >> 2));
    uint32_t gcur = (nent.x >> kEntGroupShift) & 0xFFu;
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
      const uint32_t ents[4] = {nent.x, nent.y, nent.z, nent.w};
      const uint32_t rows[4] = {nrow.x, nrow.y, nrow.z, nrow.w};
      if (e + 4 < e1) {   // the next batch's entries load under this batch's rows
        nent = __ldg(ent4p + ((e + 4) >> 2));
        nrow = __ldg(row4p + ((e + 4) >> 2));
      }
      tup_batch_c128<4, KA, PP>(xr[r], pk, dim_dn, ents, rows, coefS, sum, gcur, acc[r]);
    }
    if (e < e1) {   // the last 1-3 entries (uniform over the block)
      const uint32_t ents[4] = {nent.x, nent.y, nent.z, nent.w};
      const uint32_t rows[4] = {nrow.x, nrow.y, nrow.z, nrow.w};
      const int nb = e1 - e;
      if (nb == 1)
        tup_batch_c128<1, KA, PP>(xr[r], pk, dim_dn, ents, rows, coefS, sum, gcur, acc[r]);
      else if (nb == 2)
        tup_batch_c128<2, KA, PP>(xr[r], pk, dim_dn, ents, rows, coefS, sum, gcur, acc[r]);
      else
        tup_batch_c128<3, KA, PP>(xr[r], pk, dim_dn, ents, rows, coefS, sum, gcur, acc[r]);
    }
    const C c = coefS[gcur];
#pragma unroll
    for (int k = 0; k < 2 * KA; ++k) cmac(acc[r][k], c, sum[k]);
  }
}

template <typename R, int NR, int PP, int KA, bool VEC, int NT = kApplyThreads>
__device__ __forceinline__ void tup_chunk(const SectorDev& sd, const typename C2T<R>::T* x,
                                          const typename C2T<R>::T* coefS, const float4* coefQ,
                                          const int (&urow)[NR], int nrows, int pc, int npairs,
                                          int dim_dn,
                                          typename C2T<R>::T (&acc)[NR][2 * PP]) {
  const typename C2T<R>::T* xr[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) xr[r] = x;
  if constexpr (sizeof(R) == 4)
    tup_chunk_c64<NR, PP, KA, VEC, NT>(sd, xr, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
  else
    tup_chunk_c128<NR, PP, KA, NT>(sd, xr, coefS, urow, nrows, pc, npairs, dim_dn, acc);
}

// The same for multi-vector blocks: row r of the block is row u of the
// vector at xr[r].  The rows walk u's entry list one after the other (the
// list, its source offsets and coefficient slots are L1 hits after the
// first row), which keeps the accumulators of one row live at a time.
template <typename R, int NR, int PP, int KA, bool VEC, int NT>
__device__ __forceinline__ void tup_chunk_mv(const SectorDev& sd,
                                             const typename C2T<R>::T* const (&xr)[NR],
                                             const typename C2T<R>::T* coefS, const float4* coefQ,
                                             int u, int nrows, int pc, int npairs, int dim_dn,
                                             typename C2T<R>::T (&acc)[NR][2 * PP]) {
  int urow[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) urow[r] = u;
  if constexpr (sizeof(R) == 4)
    tup_chunk_c64<NR, PP, KA, VEC, NT>(sd, xr, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
  else
    tup_chunk_c128<NR, PP, KA, NT>(sd, xr, coefS, urow, nrows, pc, npairs, dim_dn, acc);
}

// The reduced Re<x_j, w> of one vector: j >= 1, alpha_j = Re h_jj of
// Algorithm 6 (H is Hermitian: the imaginary part of <v_j, w> is rounding);
// j == -1, the energy <x_1, H x_1> / Ns at this step.
__device__ __forceinline__ void apply_dot_result(LanczosState* st, double* out_energy, int j,
                                                 double re, int Ns) {
  if (j >= 1) {
    st->alpha[j] = re * st->inv_scale[j];
    if (!isfinite(re)) {
      st->status = 7; st->stopped = 1; st->m_eff = j > 1 ? j - 1 : 1;
    }
  } else {
    if (out_energy) out_energy[st->step] = re / Ns;
  }
}

// Shared-memory bytes in front of the TMA ring / end of the apply's dynamic
// shared memory: the tile, the group coefficients, and for complex64 the
// signed coefficient quads of the T_up gathers (16-byte aligned).
__host__ __device__ inline size_t apply_coef_end(int max_dim_dn, int nr, int n_groups, bool fp64) {
  const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
  size_t off = ((size_t)(max_dim_dn + kZeroCols) * nr + (size_t)n_groups) * csz;
  if (!fp64) off = ((off + 15) & ~(size_t)15) + (size_t)(1 + 2 * n_groups) * sizeof(float4);
  return off;
}

// One CTA (NT threads: 256, or 512 for a row pass on long rows) processes NR
// rows of one vector, the rows of its
// ApplyBlock (consecutive entries of the block order the host chose).  The
// rows are staged in shared memory column by column (TileIO),
// followed by eight zero columns that empty ELL slots read.  Thread t owns
// the column pairs p = pc + t + k*NT (k < PP) of every chunk pc, so a warp
// covers 64 consecutive columns.
//  * T_dn (within a row): the warp walks the flat slot list of its 64-column
//    ELL tile (slots grouped by bond group, trip count uniform over the
//    warp), each lane loading the two entries of its columns per slot and
//    gathering the NR row values of each source column from the tile; the
//    signed values of a group are summed and multiplied by the group
//    coefficient once.
//  * T_up (across rows): the padded entry list of row u is uniform over the
//    block; four entries at a time, each a coalesced pair load of the source
//    row per k, all in flight before they are used (tup_chunk).
//  * Epilogue: the diagonal U * popcount(up & dn) (+ on-site energies) times
//    the staged x joins the sums, w = s_j acc - beta_{j-1} s_{j-1} x_{j-1} is
//    stored in pairs, and the partial of Re<x_j, w> is accumulated.
template <typename R, int NR, int PP, bool VEC, int MINB, bool SPLIT, int TMAS, int NT, bool MV>
__global__ void __launch_bounds__(TMAS ? NT + 32 : NT, MINB)
k_apply(BatchArgs a, int j) {
  constexpr bool TMA = TMAS > 0;       // TMAS: ring stages of the TMA configurations
  constexpr uint32_t S = TMAS > 0 ? (uint32_t)TMAS : 1u;
  using C = typename C2T<R>::T;
  using TIO = TileIO<C, NR>;
  constexpr int T = NT;                      // consumer threads (all threads without TMA)
  constexpr uint32_t kSlotBytes = (uint32_t)(T * PP * 2 * sizeof(C));   // one chunk of a row
  static_assert(!(TMA && SPLIT), "the TMA ring serves the one-kernel T_up");
  static_assert(!MV || (!TMA && !SPLIT), "multi-vector blocks use the one-kernel gathers");
  static_assert((NT / 32 + (TMA ? 1 : 0)) * (MV ? NR : 1) <= 64, "reduction scratch");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[64];
  __shared__ int flag;
  __shared__ int tma_err;

  // One vector: the block's rows ab.row[0 .. nrows) of vector ab.vec.
  // Multi-vector (MV): row ab.row0 of the vectors ab.row[0 .. nrows), all of
  // one sector; every block of such a subgroup lists the same vectors, and
  // ab.vec, the first of them, holds the subgroup's block range and
  // reduction counter.
  const ApplyBlock ab = a.apply_map[blockIdx.x];
  const VecDev vd = a.vec[ab.vec];
  LanczosState* st = a.st + ab.vec;
  const int nrows = ab.nrows;
  bool rdone[NR];   // MV: rows whose vector has finished this step's Lanczos
  if constexpr (MV) {
    bool all = true;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      rdone[r] = r >= nrows || (j >= 1 && lanczos_done(a.st + ab.row[r], j));
      all = all && rdone[r];
    }
    if (all) return;   // uniform over the subgroup's blocks
  } else {
    if (j >= 1 && lanczos_done(st, j)) return;   // uniform over the vector's blocks
#pragma unroll
    for (int r = 0; r < NR; ++r) rdone[r] = false;
  }
  const SectorDev sd = a.sec[vd.sector];
  const int dim_dn = sd.dim_dn;
  const int npairs = (dim_dn + 1) >> 1;
  int urow[NR];   // the block's rows (padding slots repeat the first row)
#pragma unroll
  for (int r = 0; r < NR; ++r) urow[r] = MV ? ab.row0 : (r < nrows ? ab.row[r] : ab.row[0]);
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  C* tile = reinterpret_cast<C*>(smem_raw);              // [max_dim_dn + kZeroCols][NR]
  C* coefS = tile + (size_t)(a.max_dim_dn + kZeroCols) * NR;   // [n_groups]
  // complex64: signed coefficient quads of the T_up gathers, [1 + 2 n_groups]
  float4* coefQ = reinterpret_cast<float4*>(
      smem_raw + ((((size_t)(a.max_dim_dn + kZeroCols) * NR + (size_t)a.n_groups) * sizeof(C) + 15) &
                  ~(size_t)15));
  // TMA configurations: ring of S row chunks (128-byte aligned after
  // the coefficients), then S full and S empty mbarriers
  char* ring = nullptr;
  uint64_t* full = nullptr;
  uint64_t* empty = nullptr;
  if constexpr (TMA) {
    size_t off = apply_coef_end(a.max_dim_dn, NR, a.n_groups, sizeof(R) == 8);
    off = (off + 127) & ~(size_t)127;
    ring = reinterpret_cast<char*>(smem_raw) + off;
    full = reinterpret_cast<uint64_t*>(ring + (size_t)S * kSlotBytes);
    empty = full + S;
    if (tid == 0) {
      for (int q = 0; q < S; ++q) {
        mbar_init(full + q, 1);
        mbar_init(empty + q, T / 32);
      }
      tma_err = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
  }

  const void* cbase;
  if (j >= 1) cbase = static_cast<const char*>(a.coefs) + (size_t)st->step * a.n_groups * sizeof(C);
  else if (j == 0) cbase = a.coefs;
  else cbase = static_cast<const char*>(a.coefs_obs) + (size_t)st->step * a.n_groups * sizeof(C);
  for (int g = tid; g < a.n_groups; g += T) coefS[g] = reinterpret_cast<const C*>(cbase)[g];
  if constexpr (sizeof(R) == 4) {
    for (int i = tid; i <= 2 * a.n_groups; i += T) {
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i > 0) {
        const float2 c = reinterpret_cast<const float2*>(cbase)[(i - 1) >> 1];
        const float sg = ((i - 1) & 1) ? -1.f : 1.f;
        q = make_float4(sg * c.x, sg * c.x, sg * c.y, sg * c.y);
      }
      coefQ[i] = q;
    }
  }

  const C* x = static_cast<const C*>(j >= 1 ? xptr(vd, j, sizeof(C)) : vd.x1);
  const C* xp = (j >= 2) ? static_cast<const C*>(xptr(vd, j - 1, sizeof(C))) : nullptr;
  C* w = static_cast<C*>(vd.w);
  const R s_in = (j >= 1) ? (R)st->inv_scale[j] : (R)1;
  const R s_prev = (j >= 2) ? (R)(st->beta[j - 1] * st->inv_scale[j - 1]) : (R)0;
  const R U = (R)a.U;
  // per-row vectors (one vector: all rows alike)
  const C* xr[NR];
  const C* xpr[NR];
  C* wr[NR];
  R sinr[NR], sprevr[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    if constexpr (MV) {
      const int vi = ab.row[r < nrows ? r : 0];
      const VecDev& vr = a.vec[vi];
      const LanczosState* sr = a.st + vi;
      xr[r] = static_cast<const C*>(j >= 1 ? xptr(vr, j, sizeof(C)) : vr.x1);
      xpr[r] = (j >= 2) ? static_cast<const C*>(xptr(vr, j - 1, sizeof(C))) : nullptr;
      wr[r] = static_cast<C*>(vr.w);
      sinr[r] = (j >= 1) ? (R)sr->inv_scale[j] : (R)1;
      sprevr[r] = (j >= 2) ? (R)(sr->beta[j - 1] * sr->inv_scale[j - 1]) : (R)0;
    } else {
      xr[r] = x; xpr[r] = xp; wr[r] = w; sinr[r] = s_in; sprevr[r] = s_prev;
    }
  }

  // ---- stage the NR rows column by column, one column per thread and
  // iteration (consecutive lanes write consecutive tile columns: no bank
  // conflicts in any TileIO layout), four columns' loads in flight; the
  // columns dim_dn .. dim_dn + 7 are the zero columns empty ELL slots read.
  // The staged rows and the T_up row gathers are read through L2 only
  // (ld.global.cg), which leaves the L1 to the ELL entries.
  if (!TMA || tid < T) {
    const int ncol = dim_dn + kZeroCols;
#pragma unroll 4
    for (int d = tid; d < ncol; d += T) {
      C v[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r)
        v[r] = (r < nrows && d < dim_dn) ? __ldcg(xr[r] + (size_t)urow[r] * dim_dn + d) : czero<C>();
      TIO::store(tile, d, v);
    }
  }
  uint32_t uw[NR];
  R eu[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int u = urow[r];
    uw[r] = __ldg(sd.up_word + u);
    eu[r] = sd.up_eps ? (R)__ldg(sd.up_eps + u) : (R)0;
  }
  __syncthreads();

  double dot_d = 0.0;
  double dd_r[NR];   // MV: per vector
#pragma unroll
  for (int r = 0; r < NR; ++r) dd_r[r] = 0.0;
  uint32_t cidx = 0;     // T_up entries consumed so far (TMA ring position)
  if (TMA && tid >= T) {
    // ---- producer warp (TMA configurations): one elected lane issues the
    // row chunk of every T_up entry, chunk by chunk and row by row, in the
    // order the consumers read them
    if constexpr (TMA) {
      if (lane == 0) {
        uint32_t idx = 0;
        bool ok = true;
        for (int pc = 0; pc < npairs && ok; pc += T * PP) {
          const int np_chunk = min(T * PP, npairs - pc);
          const uint32_t bytes = (uint32_t)np_chunk * 2u * (uint32_t)sizeof(C);
          for (int r = 0; r < nrows && ok; ++r) {
            const int e0 = __ldg(sd.up_off + urow[r]), e1 = __ldg(sd.up_off + urow[r] + 1);
            for (int e = e0; e < e1; ++e, ++idx) {
              const uint32_t q = idx % S;
              // test hook: stop before this copy, as a stalled copy engine
              // would (no copy of this block is left in flight afterwards)
              if ((int)idx == a.tma_withhold) {
                ok = false;
                break;
              }
              if (idx >= (uint32_t)S &&
                  !mbar_wait(empty + q, ((idx / S) - 1u) & 1u, &tma_err, a.wait_limit)) {
                ok = false;
                break;
              }
              const uint32_t src = __ldg(sd.up_ent + e) & kEntRankMask;
              const char* g = reinterpret_cast<const char*>(x) +
                              ((size_t)src * dim_dn + 2 * (size_t)pc) * sizeof(C);
              mbar_arrive_expect_tx(full + q, bytes);
              tma_bulk_g2s(ring + (size_t)q * kSlotBytes, g, bytes, full + q);
            }
          }
        }
        if (!ok) {
          st->status = kStatusTimeout;
          // wait (bounded, ignoring the flag) for the copies still in flight
          const uint32_t first = idx > (uint32_t)S ? idx - S : 0u;
          for (uint32_t k = first; k < idx; ++k)
            for (uint32_t it = 0; it < a.wait_limit; ++it)
              if (mbar_try_wait(full + k % S, (k / S) & 1u)) break;
        }
      }
      __syncwarp();
    }
  } else
  for (int pc = 0; pc < npairs; pc += T * PP) {
    C acc[NR][2 * PP];   // off-diagonal sums; the diagonal joins in the epilogue
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int k = 0; k < 2 * PP; ++k) acc[r][k] = czero<C>();
    // ---- T_dn through the 64-column ELL tiles: flat slot list (grouped by
    // bond group, uniform over the warp), two slots of entries and their
    // tile gathers in flight, coefficient applied when the group changes.
    // One 32-bit word per lane and slot packs the lane's two entries as
    // 15-bit column units plus sign bits (TileIO::unpack); the slot groups
    // are read two at a time (tiles hold even slot counts).  The entries are
    // loaded two iterations (four slots) ahead of their gathers: the ELL
    // does not stay in L1, and its L2 latency was the exposed one
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int pw0 = pc + (tid - lane) + k * T;     // first pair of the warp
      if (pw0 < npairs) {                             // uniform over the warp
        const int tw = pw0 >> 5;
        const int q0 = __ldg(sd.dn_tslot_off + tw), q1 = __ldg(sd.dn_tslot_off + tw + 1);
        const uint32_t* ellp = TIO::ellp_for(sd.dn_ellp32, sd.dn_ellpr) + lane;
        const uint2* grp2 = reinterpret_cast<const uint2*>(sd.dn_slot_grp);
        C s0v[NR], s1v[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) { s0v[r] = czero<C>(); s1v[r] = czero<C>(); }
        uint32_t na = 0u, nb = 0u, nc = 0u, nd = 0u;
        uint2 ng = make_uint2(0u, 0u), nh = ng;
        if (q0 < q1) {
          na = __ldg(ellp + (size_t)q0 * 32);
          nb = __ldg(ellp + (size_t)(q0 + 1) * 32);
          ng = __ldg(grp2 + (q0 >> 1));
        }
        if (q0 + 2 < q1) {
          nc = __ldg(ellp + (size_t)(q0 + 2) * 32);
          nd = __ldg(ellp + (size_t)(q0 + 3) * 32);
          nh = __ldg(grp2 + ((q0 + 2) >> 1));
        }
        uint32_t gcur = ng.x;
        for (int q = q0; q < q1; q += 2) {
          const uint32_t ea = na, eb = nb;
          const uint2 gg = ng;
          na = nc; nb = nd; ng = nh;
          if (q + 4 < q1) {
            nc = __ldg(ellp + (size_t)(q + 4) * 32);
            nd = __ldg(ellp + (size_t)(q + 5) * 32);
            nh = __ldg(grp2 + ((q + 4) >> 1));
          }
          uint32_t oa0, oa1, ob0, ob1;
          R ga0, ga1, gb0, gb1;
          TIO::template unpack<R>(ea, oa0, oa1, ga0, ga1);
          TIO::template unpack<R>(eb, ob0, ob1, gb0, gb1);
          C a0[NR], a1[NR], b0[NR], b1[NR];
          TIO::load_off(tile, oa0, a0);
          TIO::load_off(tile, oa1, a1);
          TIO::load_off(tile, ob0, b0);
          TIO::load_off(tile, ob1, b1);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t g = half ? gg.y : gg.x;
            if (g != gcur) {                            // uniform over the warp
              const C c = coefS[gcur];
#pragma unroll
              for (int r = 0; r < NR; ++r) {
                cmac(acc[r][2 * k], c, s0v[r]);
                cmac(acc[r][2 * k + 1], c, s1v[r]);
                s0v[r] = czero<C>();
                s1v[r] = czero<C>();
              }
              gcur = g;
            }
            const R g0 = half ? gb0 : ga0, g1 = half ? gb1 : ga1;
#pragma unroll
            for (int r = 0; r < NR; ++r) {
              cax(s0v[r], g0, half ? b0[r] : a0[r]);
              cax(s1v[r], g1, half ? b1[r] : a1[r]);
            }
          }
        }
        if (q0 < q1) {
          const C c = coefS[gcur];
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            cmac(acc[r][2 * k], c, s0v[r]);
            cmac(acc[r][2 * k + 1], c, s1v[r]);
          }
        }
      }
    }
    // per-thread pair bases of this chunk
    bool pvalid[PP];
#pragma unroll
    for (int k = 0; k < PP; ++k) pvalid[k] = pc + tid + k * T < npairs;
    // ---- split apply: the column pass stored (T_up x) in w; add its rows
    if constexpr (SPLIT) {
      C tv[NR][2 * PP];
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < PP; ++k) {
          if (r < nrows && pvalid[k])
            load_pair<C, VEC, true>(w + (size_t)urow[r] * dim_dn, pc + tid + k * T, dim_dn,
                                    tv[r][2 * k], tv[r][2 * k + 1]);
          else { tv[r][2 * k] = czero<C>(); tv[r][2 * k + 1] = czero<C>(); }
        }
#pragma unroll
      for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < 2 * PP; ++k) {
          acc[r][k].x += tv[r][k].x;
          acc[r][k].y += tv[r][k].y;
        }
    }
    // ---- T_up through the TMA ring: the row chunk of each entry (CSR order,
    // sorted by group) waits in the next ring slot; read the thread's pairs,
    // release the slot, sum by group
    if constexpr (TMA) {
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (r < nrows) {
          const int e0 = __ldg(sd.up_off + urow[r]), e1 = __ldg(sd.up_off + urow[r] + 1);
          C sum[2 * PP];
#pragma unroll
          for (int k = 0; k < 2 * PP; ++k) sum[k] = czero<C>();
          uint32_t nent = e0 < e1 ? __ldg(sd.up_ent + e0) : 0u;
          uint32_t gcur = (nent >> kEntGroupShift) & 0xFFu;
          for (int e = e0; e < e1; ++e, ++cidx) {
            const uint32_t ent = nent;
            if (e + 1 < e1) nent = __ldg(sd.up_ent + e + 1);   // next entry under this one
            const uint32_t q = cidx % S;
            const bool ready = mbar_wait(full + q, (cidx / S) & 1u, &tma_err, a.wait_limit);
            const char* slot = ring + (size_t)q * kSlotBytes;
            C v[2 * PP];
#pragma unroll
            for (int k = 0; k < PP; ++k) {
              if (ready && pvalid[k]) {
                if constexpr (sizeof(C) == 8) {
                  const float4 f = *reinterpret_cast<const float4*>(slot + (size_t)(tid + k * T) * 16);
                  v[2 * k].x = f.x; v[2 * k].y = f.y; v[2 * k + 1].x = f.z; v[2 * k + 1].y = f.w;
                } else {
                  const C* pr = reinterpret_cast<const C*>(slot) + 2 * (size_t)(tid + k * T);
                  v[2 * k] = pr[0];
                  v[2 * k + 1] = pr[1];
                }
              } else {
                v[2 * k] = czero<C>();
                v[2 * k + 1] = czero<C>();
              }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty + q);
            const uint32_t g = (ent >> kEntGroupShift) & 0xFFu;
            if (g != gcur) {                              // uniform over the block
              const C c = coefS[gcur];
#pragma unroll
              for (int k = 0; k < 2 * PP; ++k) {
                cmac(acc[r][k], c, sum[k]);
                sum[k] = czero<C>();
              }
              gcur = g;
            }
            const R sg = sign_of<R>(ent);
#pragma unroll
            for (int k = 0; k < 2 * PP; ++k) cax(sum[k], sg, v[k]);
          }
          if (e0 < e1) {
            const C c = coefS[gcur];
#pragma unroll
            for (int k = 0; k < 2 * PP; ++k) cmac(acc[r][k], c, sum[k]);
          }
        }
      }
    }
    // ---- T_up: the padded entry lists of the rows (uniform over the block);
    // versioned on how many column-pair groups of this chunk hold valid pairs
    if constexpr (MV) {
      if (PP > 1 && pc + (PP - 1) * T < npairs)
        tup_chunk_mv<R, NR, PP, PP, VEC, NT>(sd, xr, coefS, coefQ, urow[0], nrows, pc, npairs,
                                              dim_dn, acc);
      else
        tup_chunk_mv<R, NR, PP, 1, VEC, NT>(sd, xr, coefS, coefQ, urow[0], nrows, pc, npairs,
                                             dim_dn, acc);
    } else if constexpr (!SPLIT && !TMA) {
      if (PP > 1 && pc + (PP - 1) * T < npairs)
        tup_chunk<R, NR, PP, PP, VEC, NT>(sd, x, coefS, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
      else
        tup_chunk<R, NR, PP, 1, VEC, NT>(sd, x, coefS, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
    }
    // ---- epilogue: previous-vector loads first, then scale, subtract, store
    R dot_acc = (R)0;
    R dacc_r[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) dacc_r[r] = (R)0;
    {
    C pv[NR][2 * PP];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int k = 0; k < PP; ++k) {
        const int p = pc + tid + k * T;
        if (xpr[r] && r < nrows && p < npairs)
          load_pair<C, VEC, true>(xpr[r] + (size_t)urow[r] * dim_dn, p, dim_dn, pv[r][2 * k],
                                  pv[r][2 * k + 1]);
        else { pv[r][2 * k] = czero<C>(); pv[r][2 * k + 1] = czero<C>(); }
      }
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int p = pc + tid + k * T;
      if (p < npairs) {
        // diagonal U popcount(up & dn) + eps of the pair's two columns
        const int d0 = 2 * p;
        const bool has1 = d0 + 1 < dim_dn;
        const uint32_t dw0 = __ldg(sd.dn_word + d0);
        const uint32_t dw1 = has1 ? __ldg(sd.dn_word + d0 + 1) : 0u;
        const R de0 = sd.dn_eps ? (R)__ldg(sd.dn_eps + d0) : (R)0;
        const R de1 = (sd.dn_eps && has1) ? (R)__ldg(sd.dn_eps + d0 + 1) : (R)0;
        C xa[NR], xb[NR];
        TIO::load(tile, d0, xa);
        TIO::load(tile, d0 + 1, xb);    // zero column past the end
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r < nrows) {
            const R g0 = U * (R)__popc(uw[r] & dw0) + eu[r] + de0;
            const R g1 = U * (R)__popc(uw[r] & dw1) + eu[r] + de1;
            C a0 = acc[r][2 * k], a1 = acc[r][2 * k + 1];
            a0.x += g0 * xa[r].x;
            a0.y += g0 * xa[r].y;
            a1.x += g1 * xb[r].x;
            a1.y += g1 * xb[r].y;
            C o0, o1;
            o0.x = sinr[r] * a0.x - sprevr[r] * pv[r][2 * k].x;
            o0.y = sinr[r] * a0.y - sprevr[r] * pv[r][2 * k].y;
            o1.x = sinr[r] * a1.x - sprevr[r] * pv[r][2 * k + 1].x;
            o1.y = sinr[r] * a1.y - sprevr[r] * pv[r][2 * k + 1].y;
            if (!rdone[r]) store_pair<C, VEC, true>(wr[r] + (size_t)urow[r] * dim_dn, p, dim_dn, o0, o1);
            const R dre = xa[r].x * o0.x + xa[r].y * o0.y + xb[r].x * o1.x + xb[r].y * o1.y;
            if constexpr (MV) dacc_r[r] += dre;
            else dot_acc += dre;
          }
        }
      }
    }
    }
    dot_d += (double)dot_acc;
#pragma unroll
    for (int r = 0; r < NR; ++r) dd_r[r] += (double)dacc_r[r];
  }
  if constexpr (TMA) {
    if (tma_err && tid == 0) st->status = kStatusTimeout;
  }
  if (j == 0) return;
  if constexpr (MV) {
    constexpr int KR = NR;   // Re<x_j, w> of each vector of the subgroup
    double v[KR];
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = dd_r[r];
    if (reduce_last_block<KR>(v, blockIdx.x, vd.apply_begin, vd.apply_end,
                              a.partials, a.counters + ab.vec, red, &flag)) {
      if (tid == 0)
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (!rdone[r])
            apply_dot_result(a.st + ab.row[r], a.vec[ab.row[r]].out_energy, j, v[r], a.Ns);
    }
  } else {
    double v[1] = {dot_d};   // Re<x_j, w>
    if (reduce_last_block<1>(v, blockIdx.x, vd.apply_begin, vd.apply_end,
                             a.partials, a.counters + ab.vec, red, &flag)) {
      if (tid == 0) apply_dot_result(st, vd.out_energy, j, v[0], a.Ns);
    }
  }
}

// --------------------------------------------- split apply: T_up by rows
// T_up pass of the split apply for sectors whose vector does not fit L2:
// w[u, chunk] = sum_{u'} T_up[u, u'] x[u', chunk] for the kTupRows rows of
// the block (ApplyBlock.row) over one chunk of kApplyThreads * PP column
// pairs from ApplyBlock.pc on, with the gathers of tup_chunk.  The blocks
// come chunk by chunk (append_tup_chunk), so the CTAs resident together
// gather from one chunk of columns of all rows, a working set the L2 holds
// even when the whole vector does not fit; w goes out with evict-first
// stores.  The row pass (k_apply with SPLIT) adds its rows of w.
template <typename R, int PP, bool VEC, int MINB>
__global__ void __launch_bounds__(kApplyThreads, MINB)
k_apply_tup(BatchArgs a, int j) {
  using C = typename C2T<R>::T;
  constexpr int T = kApplyThreads;
  constexpr int NR = kTupRows;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ApplyBlock ab = a.col_map[blockIdx.x];
  const VecDev vd = a.vec[ab.vec];
  const LanczosState* st = a.st + ab.vec;
  if (j >= 1 && lanczos_done(st, j)) return;   // uniform over the vector's blocks
  const SectorDev sd = a.sec[vd.sector];
  const int dim_dn = sd.dim_dn;
  const int npairs = (dim_dn + 1) >> 1;
  const int pc = ab.pc;
  const int nrows = ab.nrows;
  const int tid = threadIdx.x;
  int urow[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) urow[r] = r < nrows ? ab.row[r] : ab.row[0];

  // the group coefficients and (complex64) their signed quads, laid out as
  // in k_apply with an empty tile
  C* coefS = reinterpret_cast<C*>(smem_raw);
  float4* coefQ = reinterpret_cast<float4*>(
      smem_raw + (((size_t)a.n_groups * sizeof(C) + 15) & ~(size_t)15));
  const void* cbase;
  if (j >= 1) cbase = static_cast<const char*>(a.coefs) + (size_t)st->step * a.n_groups * sizeof(C);
  else if (j == 0) cbase = a.coefs;
  else cbase = static_cast<const char*>(a.coefs_obs) + (size_t)st->step * a.n_groups * sizeof(C);
  for (int g = tid; g < a.n_groups; g += T) coefS[g] = reinterpret_cast<const C*>(cbase)[g];
  if constexpr (sizeof(R) == 4) {
    for (int i = tid; i <= 2 * a.n_groups; i += T) {
      float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i > 0) {
        const float2 c = reinterpret_cast<const float2*>(cbase)[(i - 1) >> 1];
        const float sg = ((i - 1) & 1) ? -1.f : 1.f;
        q = make_float4(sg * c.x, sg * c.x, sg * c.y, sg * c.y);
      }
      coefQ[i] = q;
    }
  }
  __syncthreads();

  const C* x = static_cast<const C*>(j >= 1 ? xptr(vd, j, sizeof(C)) : vd.x1);
  C* w = static_cast<C*>(vd.w);
  C acc[NR][2 * PP];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < 2 * PP; ++k) acc[r][k] = czero<C>();
  if (PP > 1 && pc + (PP - 1) * T < npairs)
    tup_chunk<R, NR, PP, PP, VEC>(sd, x, coefS, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
  else
    tup_chunk<R, NR, PP, 1, VEC>(sd, x, coefS, coefQ, urow, nrows, pc, npairs, dim_dn, acc);
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int p = pc + tid + k * T;
      if (r < nrows && p < npairs)
        store_pair<C, VEC, true>(w + (size_t)urow[r] * dim_dn, p, dim_dn, acc[r][2 * k],
                                 acc[r][2 * k + 1]);
    }
}

// ------------------------------------------------------- split apply: columns
// Column pass of the split apply: w[u, d] = sum_u' T_up[u, u'] x[u', d] for
// the NC = 32 bytes / sizeof(C) columns d0 .. d0 + ncols - 1 of every row u
// (4 complex64 or 2 complex128 columns).  Those columns of all dim_up rows
// are staged in shared memory in the TileIO layout with the row index u in
// the role of the column (32 bytes per u, two zero rows past the end that
// padding entries point to), then each warp walks the warp-tiled ELL of the
// up table over 64 target rows exactly like the within-row T_dn gathers.
// Reading and writing 32-byte row segments keeps the whole pass at one read
// of x and one write of w; the row pass (k_apply with SPLIT) adds the
// diagonal and T_dn and finishes the Lanczos epilogue.
template <typename R, int PP, bool VEC, int MINB, int CB, int TC>
__global__ void __launch_bounds__(TC, MINB)
k_apply_up(BatchArgs a, int j) {
  using C = typename C2T<R>::T;
  constexpr int NC = CB / (int)sizeof(C);    // columns per block (CB = 32 or 16 bytes)
  constexpr int UPR = CB / 16;               // 16-byte units per row segment
  static_assert(CB == 16 || CB == 32, "column blocks of 16 or 32 bytes");
  using TIO = TileIO<C, NC>;
  constexpr int T = TC;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const ApplyBlock cb = a.col_map[blockIdx.x];
  const VecDev vd = a.vec[cb.vec];
  const LanczosState* st = a.st + cb.vec;
  if (j >= 1 && lanczos_done(st, j)) return;   // uniform over the vector's blocks
  const SectorDev sd = a.sec[vd.sector];
  const int dim_up = sd.dim_up, dim_dn = sd.dim_dn;
  const int d0 = cb.row0, ncols = cb.nrows;
  const int npairs = (dim_up + 1) >> 1;
  const int tid = threadIdx.x;
  const int lane = tid & 31;

  C* tile = reinterpret_cast<C*>(smem_raw);               // [max_dim_up + kZeroCols][NC]
  C* coefS = tile + (size_t)(a.max_dim_up + kZeroCols) * NC;   // [n_groups]
  const void* cbase;
  if (j >= 1) cbase = static_cast<const char*>(a.coefs) + (size_t)st->step * a.n_groups * sizeof(C);
  else if (j == 0) cbase = a.coefs;
  else cbase = static_cast<const char*>(a.coefs_obs) + (size_t)st->step * a.n_groups * sizeof(C);
  for (int g = tid; g < a.n_groups; g += T) coefS[g] = reinterpret_cast<const C*>(cbase)[g];

  const C* x = static_cast<const C*>(j >= 1 ? xptr(vd, j, sizeof(C)) : vd.x1);
  C* w = static_cast<C*>(vd.w);

  // ---- stage: the 16-byte units h of the CB-byte segment of each row u;
  // unit h holds columns h*NC/UPR .. (h+1)*NC/UPR - 1, stored at byte
  // 32u + 16 (sw(u) ^ h) of the tile for 32-byte segments, at 16u for 16-byte
  // ones.  Four units per thread in flight.
  {
    char* tb = reinterpret_cast<char*>(tile);
    const int nunits = UPR * (dim_up + kZeroCols);
    for (int i0 = tid; i0 < nunits; i0 += 4 * T) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T;
        const int u = i / UPR, h = i % UPR;
        v[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < nunits && u < dim_up) {
          const C* src = x + (size_t)u * dim_dn + d0 + h * (NC / UPR);
          if constexpr (sizeof(C) == 16) {
            if (h < ncols) v[q] = __ldg(reinterpret_cast<const float4*>(src));
          } else if constexpr (VEC) {
            if (2 * h < ncols) v[q] = __ldg(reinterpret_cast<const float4*>(src));
          } else {
            if (2 * h < ncols) { const C e = src[0]; v[q].x = e.x; v[q].y = e.y; }
            if (2 * h + 1 < ncols) { const C e = src[1]; v[q].z = e.x; v[q].w = e.y; }
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * T;
        if (i < nunits) {
          const int u = i / UPR, h = i % UPR;
          const size_t off = UPR == 2 ? 32 * (size_t)u + 16 * (((u >> 2) & 1) ^ h) : 16 * (size_t)u;
          *reinterpret_cast<float4*>(tb + off) = v[q];
        }
      }
    }
  }
  __syncthreads();

  for (int pc = 0; pc < npairs; pc += T * PP) {
    C acc[NC][2 * PP];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int k = 0; k < 2 * PP; ++k) acc[c][k] = czero<C>();
#pragma unroll
    for (int k = 0; k < PP; ++k) {
      const int pw0 = pc + (tid - lane) + k * T;     // first pair of the warp
      if (pw0 < npairs) {                             // uniform over the warp
        const int tw = pw0 >> 5;
        const int q0 = __ldg(sd.up_tslot_off + tw), q1 = __ldg(sd.up_tslot_off + tw + 1);
        const uint2* ell2 =
            reinterpret_cast<const uint2*>(TIO::ell_for(sd.up_ell, sd.up_ell16, sd.up_ell16));
        C s0v[NC], s1v[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) { s0v[c] = czero<C>(); s1v[c] = czero<C>(); }
        uint32_t gcur = q0 < q1 ? __ldg(sd.up_slot_grp + q0) : 0u;
        uint2 na = make_uint2(0u, 0u), nb = na;
        uint32_t nga = 0u, ngb = 0u;
        if (q0 < q1) {
          na = __ldg(ell2 + (size_t)q0 * 32 + lane);
          nb = __ldg(ell2 + (size_t)(q0 + 1) * 32 + lane);
          nga = __ldg(sd.up_slot_grp + q0);
          ngb = __ldg(sd.up_slot_grp + q0 + 1);
        }
        for (int q = q0; q < q1; q += 2) {
          const uint2 ea = na, eb = nb;
          const uint32_t ga = nga, gb = ngb;
          if (q + 2 < q1) {
            na = __ldg(ell2 + (size_t)(q + 2) * 32 + lane);
            nb = __ldg(ell2 + (size_t)(q + 3) * 32 + lane);
            nga = __ldg(sd.up_slot_grp + q + 2);
            ngb = __ldg(sd.up_slot_grp + q + 3);
          }
          C a0[NC], a1[NC], b0[NC], b1[NC];
          TIO::load_ent(tile, ea.x, a0);
          TIO::load_ent(tile, ea.y, a1);
          TIO::load_ent(tile, eb.x, b0);
          TIO::load_ent(tile, eb.y, b1);
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t g = half ? gb : ga;
            if (g != gcur) {                            // uniform over the warp
              const C cf = coefS[gcur];
#pragma unroll
              for (int c = 0; c < NC; ++c) {
                cmac(acc[c][2 * k], cf, s0v[c]);
                cmac(acc[c][2 * k + 1], cf, s1v[c]);
                s0v[c] = czero<C>();
                s1v[c] = czero<C>();
              }
              gcur = g;
            }
            const uint2 e = half ? eb : ea;
            const R g0 = sign_of<R>(e.x), g1 = sign_of<R>(e.y);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              cax(s0v[c], g0, half ? b0[c] : a0[c]);
              cax(s1v[c], g1, half ? b1[c] : a1[c]);
            }
          }
        }
        if (q0 < q1) {
          const C cf = coefS[gcur];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            cmac(acc[c][2 * k], cf, s0v[c]);
            cmac(acc[c][2 * k + 1], cf, s1v[c]);
          }
        }
      }
    }
    // ---- store the 32-byte segment of each of the thread's rows
#pragma unroll
    for (int k = 0; k < PP; ++k) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int u = 2 * (pc + tid + k * T) + hh;
        if (u < dim_up) {
          C* dst = w + (size_t)u * dim_dn + d0;
          if constexpr (sizeof(C) == 16) {
#pragma unroll
            for (int c = 0; c < NC; ++c)
              if (c < ncols) dst[c] = acc[c][2 * k + hh];
          } else if constexpr (VEC) {
#pragma unroll
            for (int h = 0; h < NC / 2; ++h)
              if (2 * h < ncols)
                reinterpret_cast<float4*>(dst)[h] =
                    make_float4(acc[2 * h][2 * k + hh].x, acc[2 * h][2 * k + hh].y,
                                acc[2 * h + 1][2 * k + hh].x, acc[2 * h + 1][2 * k + hh].y);
          } else {
#pragma unroll
            for (int c = 0; c < NC; ++c)
              if (c < ncols) dst[c] = acc[c][2 * k + hh];
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------------ update
// x_{j+1} = w - alpha_j s_j x_j ;  beta_j = |x_{j+1}| ;  breakdown test.
// PAIR: complex64 vectors of even length are processed two elements per
// 16-byte access (chunk boundaries are multiples of 256 elements).
template <typename R, bool PAIR>
// four CTAs per SM (64 registers): the streaming loads of more warps in
// flight; measured 49.2 -> 48.7 us at Ns=14 (complex64)
__global__ void __launch_bounds__(256, 4) k_update(BatchArgs a, int j) {
  using C = typename C2T<R>::T;
  __shared__ double red[32];
  __shared__ int flag;
  const EwBlock eb = a.ew_map[blockIdx.x];
  const VecDev vd = a.vec[eb.vec];
  LanczosState* st = a.st + eb.vec;
  if (lanczos_done(st, j)) return;
  const R as = (R)(st->alpha[j] * st->inv_scale[j]);
  double nrm_d = 0.0;
  const void* pw = vd.w;
  const void* px = xptr(vd, j, sizeof(C));
  const void* pxn = xptr(vd, j + 1, sizeof(C));
  const bool aligned = (((uintptr_t)pw | (uintptr_t)px | (uintptr_t)pxn) & 15u) == 0;
  if (PAIR && aligned && (eb.begin & 1) == 0 && (eb.end & 1) == 0) {
    const float4* w = static_cast<const float4*>(pw);
    const float4* x = static_cast<const float4*>(px);
    float4* xn = static_cast<float4*>(const_cast<void*>(pxn));
    const int64_t b2 = eb.begin >> 1, e2 = eb.end >> 1;
    const float af = (float)as;
    const int bd = blockDim.x;
    // four pairs per thread and iteration: eight 16-byte loads in flight.
    // w and x_j are not read again before the combine at the end of the
    // step: evict-first loads leave x_{j+1}, whose rows the next apply
    // gathers, in L2.
    for (int64_t i0 = b2 + threadIdx.x; i0 < e2; i0 += 4 * (int64_t)bd) {
      float4 wv[4], xv[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + (int64_t)q * bd;
        if (i < e2) { wv[q] = __ldcs(w + i); xv[q] = __ldcs(x + i); }
        else { wv[q] = make_float4(0.f, 0.f, 0.f, 0.f); xv[q] = wv[q]; }
      }
      float nrm = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t i = i0 + (int64_t)q * bd;
        float4 o;
        o.x = wv[q].x - af * xv[q].x;
        o.y = wv[q].y - af * xv[q].y;
        o.z = wv[q].z - af * xv[q].z;
        o.w = wv[q].w - af * xv[q].w;
        if (i < e2) xn[i] = o;
        nrm += o.x * o.x + o.y * o.y + o.z * o.z + o.w * o.w;
      }
      nrm_d += (double)nrm;
    }
  } else {
    const C* w = static_cast<const C*>(vd.w);
    const C* x = static_cast<const C*>(xptr(vd, j, sizeof(C)));
    C* xn = static_cast<C*>(const_cast<void*>(xptr(vd, j + 1, sizeof(C))));
    R nrm = (R)0;
    int cnt = 0;
#pragma unroll 2
    for (int64_t i = eb.begin + threadIdx.x; i < eb.end; i += blockDim.x) {
      const C wv = __ldcs(w + i), xv = __ldcs(x + i);
      C o;
      o.x = wv.x - as * xv.x;
      o.y = wv.y - as * xv.y;
      xn[i] = o;
      nrm += o.x * o.x + o.y * o.y;
      if (++cnt == 8) { nrm_d += (double)nrm; nrm = (R)0; cnt = 0; }
    }
    nrm_d += (double)nrm;
  }
  double v[1] = {nrm_d};
  if (reduce_last_block<1>(v, blockIdx.x, vd.ew_begin, vd.ew_end, a.partials,
                           a.counters + eb.vec, red, &flag)) {
    if (threadIdx.x == 0) {
      const double beta = sqrt(v[0]);
      const double sc = fmax(st->scale, fabs(st->alpha[j]));
      st->beta[j] = beta;
      st->sc_at[j] = sc;
      if (!isfinite(beta)) {
        st->status = 7; st->stopped = 1; st->m_eff = j;
      } else if (beta <= a.break_tol * sc) {
        st->stopped = 1; st->m_eff = j;
      } else {
        st->inv_scale[j + 1] = 1.0 / beta;
        st->scale = fmax(sc, beta);
      }
    }
  }
}

// -------------------------------------------------------------------- expm
// 1/k for the Taylor coefficients (evaluated by the compiler)
struct InvK {
  double v[81];
};
constexpr InvK make_inv_k() {
  InvK t{};
  t.v[0] = 0.0;
  for (int k = 1; k <= 80; ++k) t.v[k] = 1.0 / (double)k;
  return t;
}
__constant__ InvK kInvK = make_inv_k();

// exp(-i tau T) e_1 for the real symmetric tridiagonal T of size n <= 64,
// one warp.  T is shifted by the centre sigma of its Gershgorin interval,
// whose half-width h bounds |T - sigma| (2-norm), and the time step is split
// into nsub pieces with rho = |tau| h / nsub <= 1/2.  Each piece is a Taylor
// series with a term count K fixed up front: the k-th term of a piece has
// norm at most rho^k / k! (the state keeps unit norm), and the terms past K
// sum to less than rho^(K+1) / (K+1)! / (1 - rho / (K+2)) <= 1e-17, below
// rounding; K <= 16 for rho <= 1/2.  No per-term norms are reduced across
// the warp.  Lane l owns rows l and l + 32.
__device__ void tridiag_expm_e1(const double* al, const double* be, int n,
                                double tau, double* yre, double* yim,
                                double* tre, double* tim) {
  const int lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  double lo = 1e300, hi = -1e300;
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(be[i - 1]) : 0.0) + (i < n - 1 ? fabs(be[i]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(full, lo, o));
    hi = fmax(hi, __shfl_xor_sync(full, hi, o));
  }
  const double sigma = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  int nsub = (int)ceil(fabs(tau) * half / 0.5);
  if (nsub < 1) nsub = 1;
  if (nsub > 4096) nsub = 4096;
  const double ts = tau / nsub;
  // the term count from the bound (uniform over the warp)
  const double rho = fabs(ts) * half;
  int K = 1;
  {
    double b = rho;   // rho^k / k!, k = 1
    for (int k = 1; k <= 78; ++k) {
      const double nb = b * rho * kInvK.v[k + 1];   // rho^(k+1) / (k+1)!
      K = k;
      if (nb <= 1e-17 * (1.0 - rho * kInvK.v[k + 2])) break;
      b = nb;
    }
  }
  // per-lane rows: shifted diagonal and off-diagonals
  double ash[2], bl[2], bu[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    ash[h] = i < n ? al[i] - sigma : 0.0;
    bl[h] = (i < n && i > 0) ? be[i - 1] : 0.0;
    bu[h] = (i < n - 1) ? be[i] : 0.0;
  }
  for (int i = lane; i < 64; i += 32) {
    yre[i] = (i == 0) ? 1.0 : 0.0;
    yim[i] = 0.0;
  }
  __syncwarp();
  for (int sub = 0; sub < nsub; ++sub) {
    for (int i = lane; i < 64; i += 32) { tre[i] = yre[i]; tim[i] = yim[i]; }
    __syncwarp();
    for (int k = 1; k <= K; ++k) {
      double nre[2] = {0.0, 0.0}, nim[2] = {0.0, 0.0};
      const double f = ts * kInvK.v[k];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < n) {
          double qr = ash[h] * tre[i];
          double qi = ash[h] * tim[i];
          if (i > 0) { qr += bl[h] * tre[i - 1]; qi += bl[h] * tim[i - 1]; }
          if (i < n - 1) { qr += bu[h] * tre[i + 1]; qi += bu[h] * tim[i + 1]; }
          // (-i f) (qr + i qi) = f qi - i f qr
          nre[h] = f * qi;
          nim[h] = -f * qr;
        }
      }
      __syncwarp();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (i < n) {
          tre[i] = nre[h]; tim[i] = nim[h];
          yre[i] += nre[h]; yim[i] += nim[h];
        }
      }
      __syncwarp();
    }
  }
  // undo the shift: multiply by exp(-i tau sigma)
  double sn, cs;
  sincos(-tau * sigma, &sn, &cs);
  for (int i = lane; i < n; i += 32) {
    const double r = yre[i], im = yim[i];
    yre[i] = r * cs - im * sn;
    yim[i] = r * sn + im * cs;
  }
  __syncwarp();
}

// ed_tridiag_expm: one warp per problem b runs tridiag_expm_e1 on
// alpha[b n ..], beta[b (n-1) ..] (n <= 64) and writes y = exp(-i tau T) e_1
// to y[b n ..] as (re, im) pairs.
__global__ void __launch_bounds__(32) k_tridiag_expm(const double* alpha, const double* beta,
                                                     int n, double tau, double* y) {
  __shared__ double al[64], be[64], yre[64], yim[64], tre[64], tim[64];
  const size_t b = blockIdx.x;
  for (int i = threadIdx.x; i < 64; i += 32) {
    al[i] = i < n ? alpha[b * n + i] : 0.0;
    be[i] = i < n - 1 ? beta[b * (n - 1) + i] : 0.0;
  }
  __syncwarp();
  tridiag_expm_e1(al, be, n, tau, yre, yim, tre, tim);
  for (int i = threadIdx.x; i < n; i += 32) {
    y[2 * (b * n + i)] = yre[i];
    y[2 * (b * n + i) + 1] = yim[i];
  }
}

// Two warps per vector: warp 0 computes y = exp(-i tau T_n) e_1, warp 1 the
// one-smaller y^(n-1) that the a-posteriori delta compares with, at the same
// time (each a chain of float64 warp operations).
__global__ void __launch_bounds__(64) k_expm(BatchArgs a) {
  __shared__ double al[64], be[64], yre[64], yim[64], pre[64], pim[64];
  __shared__ double tre[2][64], tim[2][64];
  const int b = blockIdx.x;
  LanczosState* st = a.st + b;
  const VecDev vd = a.vec[b];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int conv = st->conv_m;
  if (conv > 0 && conv < st->m_eff) {
    // adaptive exit at step conv: its check left y^(conv) and delta
    if (warp != 0) return;
    const int n = conv;
    for (int i = lane; i < n; i += 32) {
      const double f = st->beta0 * st->inv_scale[i + 1];
      st->comb_re[i + 1] = f * st->yprev_re[i];
      st->comb_im[i + 1] = f * st->yprev_im[i];
    }
    __syncwarp();
    if (lane == 0) {
      st->m_eff = n;
      st->delta = st->conv_delta;
      if (vd.out_delta) vd.out_delta[st->step] = st->conv_delta;
      if (vd.out_meff) vd.out_meff[st->step] = n;
    }
    return;
  }
  const int n = st->m_eff;
  for (int i = threadIdx.x; i < 64; i += 64) {
    al[i] = i < n ? st->alpha[i + 1] : 0.0;
    be[i] = i < n - 1 ? st->beta[i + 1] : 0.0;
  }
  __syncthreads();
  if (warp == 0) tridiag_expm_e1(al, be, n, a.tau, yre, yim, tre[0], tim[0]);
  else if (n > 1) tridiag_expm_e1(al, be, n - 1, a.tau, pre, pim, tre[1], tim[1]);
  __syncthreads();
  if (warp != 0) return;
  double delta = 0.0;
  if (n > 1) {
    double dn = 0.0, yn = 0.0;
    for (int i = lane; i < n; i += 32) {
      const double pr = i < n - 1 ? pre[i] : 0.0, pi = i < n - 1 ? pim[i] : 0.0;
      dn += (yre[i] - pr) * (yre[i] - pr) + (yim[i] - pi) * (yim[i] - pi);
      yn += yre[i] * yre[i] + yim[i] * yim[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      dn += __shfl_xor_sync(0xffffffffu, dn, o);
      yn += __shfl_xor_sync(0xffffffffu, yn, o);
    }
    delta = sqrt(dn / yn);
  }
  for (int i = lane; i < n; i += 32) {
    const double f = st->beta0 * st->inv_scale[i + 1];
    st->comb_re[i + 1] = f * yre[i];
    st->comb_im[i + 1] = f * yim[i];
  }
  if (lane == 0) {
    st->delta = delta;
    if (vd.out_delta) vd.out_delta[st->step] = delta;
    if (vd.out_meff) vd.out_meff[st->step] = n;
  }
}

// Adaptive exit of Algorithm 6 after Lanczos step j (one warp per vector):
// y^(j) = exp(-i tau T_j) e_1, delta = |y^(j) - y^(j-1)| / |y^(j)| against the
// previous check's y (zero-padded; none at j = 1), epsilon = min(1 + |y|,
// delta / (1 - delta) |y|) for delta < 1, else 1 + |y|; the step converges
// when epsilon < eps_tol or beta_j < eps_tol * (the breakdown scale seen by
// step j).  Runs on a side stream while pass j + 1 proceeds; it reads only
// scalars of steps <= j, and writes yprev, conv_delta and conv_m.
__global__ void __launch_bounds__(32) k_conv_check(BatchArgs a, int j) {
  __shared__ double al[64], be[64], yre[64], yim[64], tre[64], tim[64];
  LanczosState* st = a.st + blockIdx.x;
  const int lane = threadIdx.x;
  if (!(st->eps_tol > 0.0) || st->conv_m > 0 || st->m_eff <= j || j >= st->m) return;
  const int n = j;
  for (int i = lane; i < 64; i += 32) {
    al[i] = i < n ? st->alpha[i + 1] : 0.0;
    be[i] = i < n - 1 ? st->beta[i + 1] : 0.0;
  }
  __syncwarp();
  tridiag_expm_e1(al, be, n, a.tau, yre, yim, tre, tim);
  double dn = 0.0, yn = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double pr = i < n - 1 ? st->yprev_re[i] : 0.0;
    const double pi = i < n - 1 ? st->yprev_im[i] : 0.0;
    dn += (yre[i] - pr) * (yre[i] - pr) + (yim[i] - pi) * (yim[i] - pi);
    yn += yre[i] * yre[i] + yim[i] * yim[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
    yn += __shfl_xor_sync(0xffffffffu, yn, o);
  }
  __syncwarp();
  for (int i = lane; i < n; i += 32) {
    st->yprev_re[i] = yre[i];
    st->yprev_im[i] = yim[i];
  }
  __syncwarp();
  if (lane == 0) {
    const double ny = sqrt(yn);
    const double delta = sqrt(dn) / ny;
    const double eps = delta < 1.0 ? fmin(1.0 + ny, delta / (1.0 - delta) * ny) : 1.0 + ny;
    if (eps < st->eps_tol || st->beta[j] < st->eps_tol * st->sc_at[j]) {
      st->conv_delta = delta;
      __threadfence();
      *(volatile int*)&st->conv_m = j;
    }
  }
}

// ------------------------------------------------------ combine / observe
// psi <- sum_j comb_j x_j (in place over x_1), fused with |psi|^2 and
// sum_k w_d[k] |psi_k|^2 (Sec. 3.5), then the per-step bookkeeping.
// In float32 the dominant coefficient c_1 is split hi + lo and its product is
// added last, which keeps the rounding of c_1 out of |psi| (the norm would
// otherwise drift by ~1e-7 per step).  Every product is accumulated by a
// chain of fused multiply-adds into p (cmac): when c_1 x was rounded on its
// own first, as in p + (a b - c d), the rounding errors of the many equal
// amplitudes of a symmetric state added up coherently and |psi|^2 drifted
// by 1-5e-8 per step, with a sign that depends on tau.
template <typename R, typename C>
__device__ __forceinline__ C combine_one(const C* cf, C cf_lo, int n, const C* V,
                                         int64_t D, int64_t i, C x) {
  C p = czero<C>();
  cmac(p, cf_lo, x);
#pragma unroll 4
  for (int jj = 1; jj < n; ++jj) cmac(p, cf[jj], V[(size_t)(jj - 1) * D + i]);
  cmac(p, cf[0], x);
  return p;
}

// Eight 16-byte streaming loads (evict-first) issued together: four pairs
// each of two Krylov vectors (element offsets o[q] from bases a and b).
__device__ __forceinline__ void ld8_stream(const float4* a, const float4* b,
                                           const int64_t (&o)[4], float4 (&va)[4],
                                           float4 (&vb)[4]) {
  asm volatile(
      "ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%32];\n\t"
      "ld.global.cs.v4.f32 {%4, %5, %6, %7}, [%33];\n\t"
      "ld.global.cs.v4.f32 {%8, %9, %10, %11}, [%34];\n\t"
      "ld.global.cs.v4.f32 {%12, %13, %14, %15}, [%35];\n\t"
      "ld.global.cs.v4.f32 {%16, %17, %18, %19}, [%36];\n\t"
      "ld.global.cs.v4.f32 {%20, %21, %22, %23}, [%37];\n\t"
      "ld.global.cs.v4.f32 {%24, %25, %26, %27}, [%38];\n\t"
      "ld.global.cs.v4.f32 {%28, %29, %30, %31}, [%39];"
      : "=f"(va[0].x), "=f"(va[0].y), "=f"(va[0].z), "=f"(va[0].w), "=f"(va[1].x),
        "=f"(va[1].y), "=f"(va[1].z), "=f"(va[1].w), "=f"(va[2].x), "=f"(va[2].y),
        "=f"(va[2].z), "=f"(va[2].w), "=f"(va[3].x), "=f"(va[3].y), "=f"(va[3].z),
        "=f"(va[3].w), "=f"(vb[0].x), "=f"(vb[0].y), "=f"(vb[0].z), "=f"(vb[0].w),
        "=f"(vb[1].x), "=f"(vb[1].y), "=f"(vb[1].z), "=f"(vb[1].w), "=f"(vb[2].x),
        "=f"(vb[2].y), "=f"(vb[2].z), "=f"(vb[2].w), "=f"(vb[3].x), "=f"(vb[3].y),
        "=f"(vb[3].z), "=f"(vb[3].w)
      : "l"(a + o[0]), "l"(a + o[1]), "l"(a + o[2]), "l"(a + o[3]), "l"(b + o[0]),
        "l"(b + o[1]), "l"(b + o[2]), "l"(b + o[3]));
}

template <typename R, bool COMBINE>
// four CTAs per SM, as k_update: 514 -> 471 us per combine at Ns=14, m=30
// (complex64), with 96 bytes of spills at 64 registers
__global__ void __launch_bounds__(256, 4) k_combine(BatchArgs a) {
  using C = typename C2T<R>::T;
  __shared__ double red[64];
  __shared__ int flag;
  __shared__ C cf[kMaxKrylov + 1];
  __shared__ C cf_lo;
  const EwBlock eb = a.ew_map[blockIdx.x];
  const VecDev vd = a.vec[eb.vec];
  LanczosState* st = a.st + eb.vec;
  const SectorDev sd = a.sec[vd.sector];
  const int n = COMBINE ? st->m_eff : 1;
  if (COMBINE) {
    for (int jj = threadIdx.x; jj < n; jj += blockDim.x) {
      cf[jj].x = (R)st->comb_re[jj + 1];
      cf[jj].y = (R)st->comb_im[jj + 1];
    }
    if (threadIdx.x == 0) {
      cf_lo.x = (R)(st->comb_re[1] - (double)(R)st->comb_re[1]);
      cf_lo.y = (R)(st->comb_im[1] - (double)(R)st->comb_im[1]);
    }
    __syncthreads();
  }
  C* x1 = static_cast<C*>(vd.x1);
  const C* V = static_cast<const C*>(vd.V);
  const int dim_dn = sd.dim_dn;
  double nd = 0.0, wd = 0.0;
  R nl = (R)0, wl = (R)0;
  int cnt = 0;
  const bool pairs = sizeof(R) == 4 && (dim_dn & 1) == 0 && (eb.begin & 1) == 0 &&
                     (eb.end & 1) == 0 && (((uintptr_t)x1 | (uintptr_t)V) & 15u) == 0 &&
                     (vd.D & 1) == 0;
  if (pairs) {
    // two elements (one row, since dim_dn is even) per 16-byte access.  The
    // block sweeps sub-chunks of 4 x 256 pairs (16 KB of every vector) one
    // Krylov vector at a time, so each vector is read in contiguous 16 KB
    // pieces; four pairs per thread accumulate in registers, two vectors'
    // loads (eight 16-byte loads) in flight.
    constexpr int Q = 4;
    float4* x4 = reinterpret_cast<float4*>(x1);
    const float4* V4 = reinterpret_cast<const float4*>(V);
    const int64_t D2 = vd.D >> 1;
    const int64_t b2 = eb.begin >> 1, e2 = eb.end >> 1;
    const int bd = blockDim.x;
    for (int64_t base = b2; base < e2; base += (int64_t)Q * bd) {
      int64_t idx[Q];
      bool ok[Q];
      float4 xv[Q], p[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        idx[q] = base + threadIdx.x + (int64_t)q * bd;
        ok[q] = idx[q] < e2;
        xv[q] = ok[q] ? x4[idx[q]] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      if (COMBINE) {
        const float2 lo = *reinterpret_cast<const float2*>(&cf_lo);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          p[q] = make_float4(0.f, 0.f, 0.f, 0.f);
          cmac4(p[q], lo, xv[q]);
        }
        // JV Krylov vectors per round, all JV x Q loads issued before their
        // products, by volatile loads at in-range indices (out-of-range
        // lanes read element e2 - 1 and drop it).  Left to the compiler, the
        // loads of one vector waited for the previous vector's products,
        // about one vector's loads were in flight per thread, and the kernel
        // ran 2.3x slower.  Accumulation order j = 1, 2, ... as in combine_one.
        constexpr int JV = 4;
        int64_t ldi[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) ldi[q] = ok[q] ? idx[q] : e2 - 1;
        int jj = 1;
        for (; jj + JV <= n; jj += JV) {
          float4 v[JV][Q];
#pragma unroll
          for (int u = 0; u < JV; u += 2) {
            const float4* Vj = V4 + (size_t)(jj + u - 1) * D2;
            ld8_stream(Vj, Vj + D2, ldi, v[u], v[u + 1]);
          }
#pragma unroll
          for (int u = 0; u < JV; ++u)
#pragma unroll
            for (int q = 0; q < Q; ++q)
              if (!ok[q]) v[u][q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < JV; ++u) {
            const float2 c = *reinterpret_cast<const float2*>(&cf[jj + u]);
#pragma unroll
            for (int q = 0; q < Q; ++q) cmac4(p[q], c, v[u][q]);
          }
        }
        for (; jj < n; ++jj) {
          const float4* Vj = V4 + (size_t)(jj - 1) * D2;
          const float2 c = *reinterpret_cast<const float2*>(&cf[jj]);
          float4 v[Q];
#pragma unroll
          for (int q = 0; q < Q; ++q)
            v[q] = ok[q] ? __ldcs(Vj + idx[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q = 0; q < Q; ++q) cmac4(p[q], c, v[q]);
        }
        const float2 c0 = *reinterpret_cast<const float2*>(&cf[0]);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          cmac4(p[q], c0, xv[q]);
          if (ok[q]) x4[idx[q]] = p[q];
        }
      } else {
#pragma unroll
        for (int q = 0; q < Q; ++q) p[q] = xv[q];
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        if (!ok[q]) continue;
        // sector indices fit 32 bits (D <= C(16,8)^2 < 2^28): 32-bit division
        const uint32_t e = 2u * (uint32_t)idx[q];
        const int u = (int)(e / (uint32_t)dim_dn);
        const int d = (int)(e - (uint32_t)u * (uint32_t)dim_dn);
        const uint32_t uwd = __ldg(sd.up_word + u);
        const R q0 = p[q].x * p[q].x + p[q].y * p[q].y, q1 = p[q].z * p[q].z + p[q].w * p[q].w;
        nl += q0 + q1;
        wl += (R)__popc(uwd & __ldg(sd.dn_word + d)) * q0 +
              (R)__popc(uwd & __ldg(sd.dn_word + d + 1)) * q1;
      }
      nd += (double)nl;
      wd += (double)wl;
      nl = wl = (R)0;
    }
  } else {
    for (int64_t i = eb.begin + threadIdx.x; i < eb.end; i += blockDim.x) {
      C p = x1[i];
      if (COMBINE) {
        p = combine_one<R, C>(cf, cf_lo, n, V, vd.D, i, p);
        x1[i] = p;
      }
      const int u = (int)((uint32_t)i / (uint32_t)dim_dn);
      const int d = (int)((uint32_t)i - (uint32_t)u * (uint32_t)dim_dn);
      const R q = p.x * p.x + p.y * p.y;
      nl += q;
      wl += (R)__popc(__ldg(sd.up_word + u) & __ldg(sd.dn_word + d)) * q;
      if (++cnt == 8) { nd += (double)nl; wd += (double)wl; nl = wl = (R)0; cnt = 0; }
    }
  }
  double v[2] = {nd + (double)nl, wd + (double)wl};
  if (reduce_last_block<2>(v, blockIdx.x, vd.ew_begin, vd.ew_end, a.partials,
                           a.counters + eb.vec, red, &flag)) {
    if (threadIdx.x == 0) {
      const double norm2 = v[0];
      const int slot = COMBINE ? st->step + 1 : st->step;
      if (vd.out_docc) vd.out_docc[slot] = v[1] / a.Ns;
      if (vd.out_norm2) vd.out_norm2[slot] = norm2;
      const double b0 = sqrt(norm2);
      if (!isfinite(b0)) st->status = 7;
      st->beta0 = b0;
      st->inv_scale[1] = b0 > 0.0 ? 1.0 / b0 : 0.0;
      st->scale = 1.0;
      st->m_eff = st->m;
      st->conv_m = 0;
      st->stopped = b0 > 0.0 && isfinite(b0) ? 0 : 1;
      if (COMBINE) st->step = st->step + 1;
    }
  }
}

// -------------------------------------------------------- fermion operator
// Element (u, d) of the target sector dim_up_dst x dim_dn_dst, at storage
// index t: row-major (t = u dim_dn + d) for spin 0 and 1, column-major
// (t = d dim_up + u, the vector stored transposed) for spin mode 2.
// (Sector indices fit 32 bits, D <= C(16,8)^2 < 2^28: 32-bit division, which
// costs a fraction of a 64-bit one.)
__device__ __forceinline__ void target_ud(int64_t t, int dim_up, int dim_dn, int spin, int& u,
                                          int& d) {
  const uint32_t t32 = (uint32_t)t;
  if (spin == 2) {
    d = (int)(t32 / (uint32_t)dim_up);
    u = (int)(t32 - (uint32_t)d * (uint32_t)dim_up);
  } else {
    u = (int)(t32 / (uint32_t)dim_dn);
    d = (int)(t32 - (uint32_t)u * (uint32_t)dim_dn);
  }
}

// out = op psi through the map of the operator's spin: spin 0 a row map
// (up spin), 1 a column map (down spin), 2 a column map with out stored
// transposed (dim_dn_dst x dim_up_dst: as a vector of the sector with the two
// spins' particle numbers swapped, whose Hamiltonian is the same).
template <typename R>
__global__ void k_fermion_op(const typename C2T<R>::T* in,
                             typename C2T<R>::T* out, int dim_dn_src,
                             int dim_up_dst, int dim_dn_dst, int spin,
                             const int32_t* map) {
  using C = typename C2T<R>::T;
  const int64_t n = (int64_t)dim_up_dst * dim_dn_dst;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int u, d;
    target_ud(t, dim_up_dst, dim_dn_dst, spin, u, d);
    const int32_t m = __ldg(map + (spin == 0 ? u : d));
    C o = czero<C>();
    if (m != 0x7FFFFFFF) {
      const int src = m & 0x7FFFFFFF;
      const C v = spin == 0 ? in[(int64_t)src * dim_dn_src + d]
                            : in[(int64_t)u * dim_dn_src + src];
      o = (m < 0) ? C{-v.x, -v.y} : v;
    }
    out[t] = o;
  }
}

// ---------------------------------------------------------------- overlaps
// <op psi | phi_b> = sum_t conj(sign(t) psi[src(t)]) phi_b[t]
template <typename R>
__global__ void __launch_bounds__(256) k_overlap(BatchArgs a, OverlapArgs o) {
  using C = typename C2T<R>::T;
  __shared__ double red[64];
  __shared__ int flag;
  const EwBlock eb = a.ew_map[blockIdx.x];
  const int64_t moff = o.map_off[eb.vec];
  if (moff < 0) return;
  const VecDev vd = a.vec[eb.vec];
  const VecDev vp = a.vec[o.psi_index];
  const SectorDev sd = a.sec[vd.sector];
  const SectorDev sp = a.sec[vp.sector];
  const int spin = o.map_spin[eb.vec];
  const int32_t* map = o.maps + moff;
  const C* phi = static_cast<const C*>(vd.x1);
  const C* psi = static_cast<const C*>(vp.x1);
  // spin mode 2: phi is stored transposed (a vector of the sector with the
  // spins' particle numbers swapped), so its storage shape is sd's and the
  // target sector of the map is sd with rows and columns exchanged
  const int dim_up_t = spin == 2 ? sd.dim_dn : sd.dim_up;
  const int dim_dn_t = spin == 2 ? sd.dim_up : sd.dim_dn;
  const int dim_dn_src = sp.dim_dn, dim_up_src = sp.dim_up;
  // mode 2 reads psi transposed: row src of psi^T is column src of psi, so
  // consecutive t (consecutive u) read consecutive elements
  const C* psiT = static_cast<const C*>(o.psiT);
  // conj(s p) f per element (s = +-1), summed in the vector precision over
  // at most 8 elements per thread and then in float64 (as the norms): in
  // complex64 a float64 product and sum per element made the kernel
  // FP64-pipe bound (0.3-0.5 TB/s)
  double ar = 0.0, ai = 0.0;
  R pr = (R)0, pi = (R)0;
  int cnt = 0;
  for (int64_t t = eb.begin + threadIdx.x; t < eb.end; t += blockDim.x) {
    int u, d;
    target_ud(t, dim_up_t, dim_dn_t, spin, u, d);
    const int32_t m = __ldg(map + (spin == 0 ? u : d));
    if (m == 0x7FFFFFFF) continue;
    const int src = m & 0x7FFFFFFF;
    const C p = spin == 0   ? psi[(int64_t)src * dim_dn_src + d]
                : spin == 2 ? psiT[(int64_t)src * dim_up_src + u]
                            : psi[(int64_t)u * dim_dn_src + src];
    const C f = phi[t];
    const R sg = m < 0 ? (R)-1 : (R)1;
    pr += sg * (p.x * f.x + p.y * f.y);
    pi += sg * (p.x * f.y - p.y * f.x);
    if (++cnt == 8) { ar += (double)pr; ai += (double)pi; pr = pi = (R)0; cnt = 0; }
  }
  ar += (double)pr;
  ai += (double)pi;
  double v[2] = {ar, ai};
  if (reduce_last_block<2>(v, blockIdx.x, vd.ew_begin, vd.ew_end, a.partials,
                           a.counters + eb.vec, red, &flag)) {
    if (threadIdx.x == 0) {
      const int step = a.st[o.psi_index].step;
      double* out = o.out + ((size_t)step * a.nvec + eb.vec) * 2;
      out[0] = v[0];
      out[1] = v[1];
    }
  }
}

// Tiled transpose of a rows x cols complex matrix through shared memory
// (32 x 32 tiles, one padding column against bank conflicts): reads and
// writes are both row-contiguous.
template <typename C>
__global__ void __launch_bounds__(256) k_transpose(const C* in, C* out, int rows, int cols) {
  __shared__ C tile[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int r = r0 + ty + k, c = c0 + tx;
    if (r < rows && c < cols) tile[ty + k][tx] = in[(size_t)r * cols + c];
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int c = c0 + ty + k, r = r0 + tx;
    if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[tx][ty + k];
  }
}

// ------------------------------------------------------ ground-state helpers
__global__ void __launch_bounds__(256)
k_multidot(const double2* V, int64_t ldV, int k, const double2* w, int64_t D,
           double2* partial) {
  // block b handles chunk [b*chunk, (b+1)*chunk); partial[b*k + i]
  extern __shared__ double2 sacc[];  // [blockDim/32][k]
  const int64_t chunk = (D + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(D, i0 + chunk);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = 0; i < k; ++i) {
    double re = 0.0, im = 0.0;
    const double2* Vi = V + (size_t)i * ldV;
    for (int64_t t = i0 + threadIdx.x; t < i1; t += blockDim.x) {
      const double2 a = Vi[t], b = w[t];
      re += a.x * b.x + a.y * b.y;
      im += a.x * b.y - a.y * b.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_down_sync(0xffffffffu, re, o);
      im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) sacc[wid * k + i] = make_double2(re, im);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int q = 0; q < nw; ++q) { re += sacc[q * k + i].x; im += sacc[q * k + i].y; }
    partial[(size_t)blockIdx.x * k + i] = make_double2(re, im);
  }
}

__global__ void k_reduce_cols(const double2* partial, int nblk, int k, double2* out) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < k; i += blockDim.x * gridDim.x) {
    double re = 0.0, im = 0.0;
    for (int b = 0; b < nblk; ++b) { re += partial[(size_t)b * k + i].x; im += partial[(size_t)b * k + i].y; }
    out[i] = make_double2(re, im);
  }
}

__global__ void k_multiaxpy(const double2* V, int64_t ldV, int k, const double2* c,
                            double2* w, int64_t D) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D;
       t += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[t];
    for (int i = 0; i < k; ++i) {
      const double2 v = V[(size_t)i * ldV + t], ci = c[i];
      acc.x -= ci.x * v.x - ci.y * v.y;
      acc.y -= ci.x * v.y + ci.y * v.x;
    }
    w[t] = acc;
  }
}

__global__ void k_combine_real(const double2* V, int64_t ldV, int k, const double* c,
                               double2* y, int64_t D) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D;
       t += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < k; ++i) {
      const double2 v = V[(size_t)i * ldV + t];
      acc.x += c[i] * v.x;
      acc.y += c[i] * v.y;
    }
    y[t] = acc;
  }
}

__global__ void __launch_bounds__(256)
k_norm_dot_partial(const double2* x, const double2* y, int64_t D, double* partial) {
  __shared__ double red[64];
  const int64_t chunk = (D + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(D, i0 + chunk);
  double v[2] = {0.0, 0.0};
  for (int64_t t = i0 + threadIdx.x; t < i1; t += blockDim.x) {
    const double2 a = x[t];
    v[0] += a.x * a.x + a.y * a.y;
    if (y) { const double2 b = y[t]; v[1] += a.x * b.x + a.y * b.y; }
  }
  block_reduce<2>(v, red);
  if (threadIdx.x == 0) { partial[2 * blockIdx.x] = v[0]; partial[2 * blockIdx.x + 1] = v[1]; }
}

__global__ void __launch_bounds__(256) k_sum_pairs(const double* partial, int nblk, double* out) {
  __shared__ double red[64];
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) { v[0] += partial[2 * b]; v[1] += partial[2 * b + 1]; }
  block_reduce<2>(v, red);
  if (threadIdx.x == 0) { out[0] = v[0]; out[1] = v[1]; }
}

__global__ void k_scale(double2* x, int64_t D, const double* s_dev, int inv_sqrt) {
  const double s = inv_sqrt ? 1.0 / sqrt(*s_dev) : *s_dev;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D;
       t += (int64_t)gridDim.x * blockDim.x) {
    x[t].x *= s;
    x[t].y *= s;
  }
}

__global__ void k_axpy_real(double2* y, const double2* x, int64_t D, const double* a_dev,
                            double a_sign) {
  const double a = a_sign * (*a_dev);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D;
       t += (int64_t)gridDim.x * blockDim.x) {
    y[t].x += a * x[t].x;
    y[t].y += a * x[t].y;
  }
}

// splitmix64 (Steele, Lea, Flood 2014) of (seed, index) -> two uniforms in
// (-1, 1) per element; the start vector only needs to overlap the ground state.
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__global__ void k_random_fill(double2* x, int64_t D, uint64_t seed) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < D;
       t += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t r1 = splitmix64(seed ^ splitmix64(2 * (uint64_t)t));
    const uint64_t r2 = splitmix64(seed ^ splitmix64(2 * (uint64_t)t + 1));
    x[t].x = ((double)(r1 >> 11) * 0x1.0p-53) * 2.0 - 1.0;
    x[t].y = ((double)(r2 >> 11) * 0x1.0p-53) * 2.0 - 1.0;
  }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_docc_sites(const typename C2T<R>::T* psi, SectorDev sd, int Ns, double* partial) {
  __shared__ double red[32 * (kMaxSites + 1)];
  const int64_t D = (int64_t)sd.dim_up * sd.dim_dn;
  const int64_t chunk = (D + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(D, i0 + chunk);
  double v[kMaxSites + 1];
#pragma unroll
  for (int i = 0; i <= kMaxSites; ++i) v[i] = 0.0;
  for (int64_t t = i0 + threadIdx.x; t < i1; t += blockDim.x) {
    const int u = (int)((uint32_t)t / (uint32_t)sd.dim_dn);
    const int d = (int)((uint32_t)t - (uint32_t)u * (uint32_t)sd.dim_dn);
    const auto p = psi[t];
    const double q = (double)p.x * p.x + (double)p.y * p.y;
    const uint32_t both = sd.up_word[u] & sd.dn_word[d];
    v[0] += __popc(both) * q;
#pragma unroll
    for (int i = 0; i < kMaxSites; ++i)
      if ((both >> i) & 1u) v[1 + i] += q;
  }
  block_reduce<kMaxSites + 1>(v, red);
  if (threadIdx.x == 0)
    for (int i = 0; i <= kMaxSites; ++i) partial[(size_t)blockIdx.x * (kMaxSites + 1) + i] = v[i];
}

__global__ void k_sum_sites(const double* partial, int nblk, int K, double* out) {
  const int i = threadIdx.x;
  if (i >= K) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * K + i];
  out[i] = s;
}

__global__ void k_convert_c128_c64(const double2* in, float2* out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = make_float2((float)in[t].x, (float)in[t].y);
}
__global__ void k_convert_c64_c128(const float2* in, double2* out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = make_double2((double)in[t].x, (double)in[t].y);
}

// ---------------------------------------------------------------- launchers
static int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  const int64_t cap = 152 * 16;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Configurations of the apply: rows per CTA (NR), column pairs per thread per
// chunk (PP) and the occupancy target (MINB CTAs per SM, which sets the
// register budget) of the row kernel; for the split apply also the pairs per
// thread and occupancy of the column pass.  The autotuner times the feasible
// ones.
struct ApplyCfg { bool fp64; int nr, pp, minb; bool split; int ppc, minbc, cb, tc; int tma; int nt; bool mv; };
// tma: 0, or the ring stages of a configuration whose T_up row chunks are
// staged by TMA
static const ApplyCfg kApplyCfgs[] = {
    {false, 4, 2, 2, false, 0, 0, 0, 0}, {false, 2, 2, 3, false, 0, 0, 0, 0},
    {false, 2, 1, 4, false, 0, 0, 0, 0}, {false, 1, 2, 2, false, 0, 0, 0, 0},
    {true, 2, 1, 2, false, 0, 0, 0, 0},  {true, 1, 1, 4, false, 0, 0, 0, 0},
    {true, 1, 1, 2, false, 0, 0, 0, 0},
    {false, 4, 2, 2, true, 1, 2, 32, 256}, {false, 2, 2, 3, true, 1, 2, 32, 256},
    {false, 2, 1, 4, true, 1, 2, 32, 256}, {false, 4, 2, 2, true, 2, 2, 32, 256},
    {true, 2, 1, 2, true, 1, 2, 32, 256},  {true, 1, 1, 4, true, 1, 2, 32, 256},
    // long columns (vectors beyond L2): 16-byte column blocks, one 512-thread
    // column CTA per SM
    {false, 1, 2, 2, true, 1, 1, 16, 512}, {true, 1, 1, 1, true, 1, 1, 16, 512},
    // one kernel with the T_up row chunks staged by TMA (a producer warp)
    {false, 2, 2, 2, false, 0, 0, 0, 0, 6}, {false, 1, 2, 2, false, 0, 0, 0, 0, 8},
    {true, 1, 1, 2, false, 0, 0, 0, 0, 6},
    // split with the row-gather T_up pass (chunk-major; vectors beyond L2):
    // chunks of 256 or 512 column pairs
    {false, 1, 2, 2, true, 1, 4, 0, 256}, {false, 1, 2, 2, true, 2, 3, 0, 256},
    // the same with a 512-thread row pass (twice the warps per SM on long rows),
    // and with two rows in one 1024-thread CTA per SM
    {false, 1, 1, 2, true, 2, 3, 0, 256, 0, 512}, {false, 2, 1, 1, true, 2, 3, 0, 256, 0, 1024},
    // multi-vector blocks (batches with several vectors in one sector): one
    // row of nr vectors per CTA (the per-vector pointers and sums need more
    // registers than configuration 1's three CTAs per SM allow)
    {false, 2, 2, 2, false, 0, 0, 0, 0, 0, 256, true}, {true, 2, 1, 2, false, 0, 0, 0, 0, 0, 256, true},
};
static const int kNumApplyCfgs = (int)(sizeof(kApplyCfgs) / sizeof(kApplyCfgs[0]));

int apply_config_count() { return kNumApplyCfgs; }
bool apply_config_info(int i, int* fp64, int* nr, int* pp, int* minb, int* split, int* tma,
                       int* mv) {
  if (i < 0 || i >= kNumApplyCfgs) return false;
  const ApplyCfg& c = kApplyCfgs[i];
  *fp64 = c.fp64;
  *nr = c.nr;
  *pp = c.pp;
  *minb = c.minb;
  *split = c.split;
  *tma = c.tma > 0;
  *mv = c.mv;
  return true;
}

std::vector<LaunchShape> apply_candidates(int max_dim_up, int max_dim_dn, bool fp64,
                                          int n_groups) {
  const size_t csz = fp64 ? sizeof(double2) : sizeof(float2);
  std::vector<LaunchShape> out;
  auto make = [&](int i) {
    const ApplyCfg& c = kApplyCfgs[i];
    LaunchShape sh;
    sh.threads = c.nt ? c.nt : kApplyThreads;
    sh.ept = c.pp;
    sh.nr = c.nr;
    sh.cfg = i;
    sh.split = c.split;
    sh.cb = c.cb;
    sh.tc = c.tc;
    sh.tma = c.tma > 0;
    sh.mv = c.mv;
    sh.smem = apply_coef_end(max_dim_dn, c.nr, n_groups, fp64);
    if (c.tma)   // 128-byte aligned ring of row chunks + full/empty mbarriers
      sh.smem = ((sh.smem + 127) & ~(size_t)127) +
                (size_t)c.tma * kApplyThreads * c.pp * 2 * csz + 2 * (size_t)c.tma * 8;
    sh.ppc = c.ppc;
    sh.smem_c = !c.split ? 0
                : c.cb == 0 ? apply_coef_end(0, 0, n_groups, fp64)   // coefficients only
                            : (size_t)(max_dim_up + kZeroCols) * c.cb + (size_t)n_groups * csz;
    return sh;
  };
  for (int i = 0; i < kNumApplyCfgs; ++i) {
    const ApplyCfg& c = kApplyCfgs[i];
    if (c.fp64 != fp64) continue;
    LaunchShape sh = make(i);
    // the CTAs per SM each kernel aims at must fit in shared memory
    if (sh.smem * (size_t)c.minb > 228 * 1024 || sh.smem > 227 * 1024) continue;
    if (c.split && (sh.smem_c * (size_t)c.minbc > 228 * 1024 || sh.smem_c > 227 * 1024)) continue;
    out.push_back(sh);
  }
  bool have_fused = false;
  for (const LaunchShape& sh : out) have_fused |= !sh.split && !sh.tma;
  if (!have_fused) {   // very long rows: one row per CTA, one CTA per SM;
    // of those entries the one with the fewest target CTAs per SM (the
    // largest register budget)
    int best = -1;
    for (int i = 0; i < kNumApplyCfgs; ++i) {
      const ApplyCfg& c = kApplyCfgs[i];
      if (c.fp64 != fp64 || c.nr != 1 || c.split || c.tma) continue;
      if (best < 0 || c.minb < kApplyCfgs[best].minb) best = i;
    }
    if (best >= 0) {
      LaunchShape sh = make(best);
      if (sh.smem <= 227 * 1024) out.push_back(sh);
    }
  }
  return out;
}

LaunchShape apply_shape(int max_dim_up, int max_dim_dn, bool fp64, int n_groups) {
  std::vector<LaunchShape> c = apply_candidates(max_dim_up, max_dim_dn, fp64, n_groups);
  if (c.empty()) {
    LaunchShape sh{};
    sh.nr = 0;   // no feasible configuration
    return sh;
  }
  return c.front();
}

template <typename R, int NR, int PP, int MINB, bool SPLIT, int PPC, int MINBC, int CB, int TC,
          int TMA, int NT, bool MV>
static cudaError_t launch_apply_t(const BatchArgs& a, int nblk, const LaunchShape& sh,
                                  int j, cudaStream_t s) {
  constexpr bool V = sizeof(R) == 4;
  constexpr int threads = TMA ? NT + 32 : NT;
  if constexpr (SPLIT && CB == 0) {
    if (sh.vec) k_apply_tup<R, PPC, V, MINBC><<<a.n_col_blocks, kApplyThreads, sh.smem_c, s>>>(a, j);
    else k_apply_tup<R, PPC, false, MINBC><<<a.n_col_blocks, kApplyThreads, sh.smem_c, s>>>(a, j);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  } else if constexpr (SPLIT) {
    if (sh.vec) k_apply_up<R, PPC, V, MINBC, CB, TC><<<a.n_col_blocks, TC, sh.smem_c, s>>>(a, j);
    else k_apply_up<R, PPC, false, MINBC, CB, TC><<<a.n_col_blocks, TC, sh.smem_c, s>>>(a, j);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (sh.vec) k_apply<R, NR, PP, V, MINB, SPLIT, TMA, NT, MV><<<nblk, threads, sh.smem, s>>>(a, j);
  else k_apply<R, NR, PP, false, MINB, SPLIT, TMA, NT, MV><<<nblk, threads, sh.smem, s>>>(a, j);
  return cudaGetLastError();
}

template <typename R, int NR, int PP, int MINB, bool SPLIT, int PPC, int MINBC, int CB, int TC,
          int TMA, int NT, bool MV>
static cudaError_t prepare_apply_t(const LaunchShape& sh) {
  constexpr bool V = sizeof(R) == 4;
  const int sm = (int)sh.smem;
  cudaError_t e = cudaFuncSetAttribute(k_apply<R, NR, PP, false, MINB, SPLIT, TMA, NT, MV>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_apply<R, NR, PP, V, MINB, SPLIT, TMA, NT, MV>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  if constexpr (SPLIT && CB == 0) {
    const int smc = (int)sh.smem_c;
    e = cudaFuncSetAttribute(k_apply_tup<R, PPC, false, MINBC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_apply_tup<R, PPC, V, MINBC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
  } else if constexpr (SPLIT) {
    const int smc = (int)sh.smem_c;
    e = cudaFuncSetAttribute(k_apply_up<R, PPC, false, MINBC, CB, TC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_apply_up<R, PPC, V, MINBC, CB, TC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smc);
  }
  return e;
}

// One switch over the configuration table for both prepare and launch.
#define ED_APPLY_CONFIGS(X)                                \
  X(0, float, 4, 2, 2, false, 1, 1, 32, 256, 0, 256, false)  \
  X(1, float, 2, 2, 3, false, 1, 1, 32, 256, 0, 256, false)  \
  X(2, float, 2, 1, 4, false, 1, 1, 32, 256, 0, 256, false)  \
  X(3, float, 1, 2, 2, false, 1, 1, 32, 256, 0, 256, false)  \
  X(4, double, 2, 1, 2, false, 1, 1, 32, 256, 0, 256, false) \
  X(5, double, 1, 1, 4, false, 1, 1, 32, 256, 0, 256, false) \
  X(6, double, 1, 1, 2, false, 1, 1, 32, 256, 0, 256, false) \
  X(7, float, 4, 2, 2, true, 1, 2, 32, 256, 0, 256, false)   \
  X(8, float, 2, 2, 3, true, 1, 2, 32, 256, 0, 256, false)   \
  X(9, float, 2, 1, 4, true, 1, 2, 32, 256, 0, 256, false)   \
  X(10, float, 4, 2, 2, true, 2, 2, 32, 256, 0, 256, false)  \
  X(11, double, 2, 1, 2, true, 1, 2, 32, 256, 0, 256, false) \
  X(12, double, 1, 1, 4, true, 1, 2, 32, 256, 0, 256, false) \
  X(13, float, 1, 2, 2, true, 1, 1, 16, 512, 0, 256, false)  \
  X(14, double, 1, 1, 1, true, 1, 1, 16, 512, 0, 256, false) \
  X(15, float, 2, 2, 2, false, 1, 1, 32, 256, 6, 256, false) \
  X(16, float, 1, 2, 2, false, 1, 1, 32, 256, 8, 256, false) \
  X(17, double, 1, 1, 2, false, 1, 1, 32, 256, 6, 256, false) \
  X(18, float, 1, 2, 2, true, 1, 4, 0, 256, 0, 256, false)   \
  X(19, float, 1, 2, 2, true, 2, 3, 0, 256, 0, 256, false)   \
  X(20, float, 1, 1, 2, true, 2, 3, 0, 256, 0, 512, false)   \
  X(21, float, 2, 1, 1, true, 2, 3, 0, 256, 0, 1024, false) \
  X(22, float, 2, 2, 2, false, 1, 1, 32, 256, 0, 256, true)  \
  X(23, double, 2, 1, 2, false, 1, 1, 32, 256, 0, 256, true)

cudaError_t prepare_apply(bool fp64, const LaunchShape& sh) {
  (void)fp64;
  if (sh.nr < 1 || sh.smem > 227 * 1024 || sh.smem_c > 227 * 1024) return cudaErrorInvalidValue;
#define X(i, R, NR, PP, MB, SP, PPC, MBC, CB, TC, TM, NT, MV) \
  case i: return prepare_apply_t<R, NR, PP, MB, SP, PPC, MBC, CB, TC, TM, NT, MV>(sh);
  switch (sh.cfg) {
    ED_APPLY_CONFIGS(X)
    default: return cudaErrorInvalidValue;
  }
#undef X
}

cudaError_t launch_apply(bool fp64, const BatchArgs& a, int nblk, const LaunchShape& sh,
                         int j, cudaStream_t s) {
  (void)fp64;
#define X(i, R, NR, PP, MB, SP, PPC, MBC, CB, TC, TM, NT, MV) \
  case i: return launch_apply_t<R, NR, PP, MB, SP, PPC, MBC, CB, TC, TM, NT, MV>(a, nblk, sh, j, s);
  switch (sh.cfg) {
    ED_APPLY_CONFIGS(X)
    default: return cudaErrorInvalidValue;
  }
#undef X
}

cudaError_t launch_update(bool fp64, const BatchArgs& a, int nblk, int j, cudaStream_t s) {
  if (fp64) k_update<double, false><<<nblk, 256, 0, s>>>(a, j);
  else k_update<float, true><<<nblk, 256, 0, s>>>(a, j);
  return cudaGetLastError();
}

cudaError_t launch_conv_check(const BatchArgs& a, int j, cudaStream_t s) {
  k_conv_check<<<a.nvec, 32, 0, s>>>(a, j);
  return cudaGetLastError();
}

cudaError_t launch_expm(const BatchArgs& a, cudaStream_t s) {
  k_expm<<<a.nvec, 64, 0, s>>>(a);
  return cudaGetLastError();
}

// Column permutation of every row of a dim_up x dim_dn matrix, from src to
// dst (the same matrix for the in-place form; either may be a pinned host
// buffer mapped into the device's address space): one CTA per row stages it
// in shared memory, then gathers dst[u][i] = src[u][g[i]], so that both the
// row's reads and its writes are coalesced (a host row crosses the host link
// once each way in whole lines).  g = order (ascending-word columns -> hop
// order: dst[u][i] = src[u][order[i]]) or its inverse (back:
// dst[u][order[i]] = src[u][i]).
template <typename C>
__global__ void __launch_bounds__(256) k_permute_cols(const C* src, C* dst, int dim_dn,
                                                      const int32_t* g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* row = reinterpret_cast<C*>(smem_raw);
  const C* sr = src + (size_t)blockIdx.x * dim_dn;
  C* dr = dst + (size_t)blockIdx.x * dim_dn;
#pragma unroll 4
  for (int d = threadIdx.x; d < dim_dn; d += blockDim.x) row[d] = sr[d];
  __syncthreads();
#pragma unroll 4
  for (int i = threadIdx.x; i < dim_dn; i += blockDim.x) dr[i] = row[__ldg(g + i)];
}

// order: the permutation (position -> rank) followed by its inverse, 2 dim_dn
// entries
static cudaError_t permute_cols(bool fp64, const void* src, void* dst, int dim_up, int dim_dn,
                                const int32_t* order, bool forward, cudaStream_t s) {
  const int32_t* g = forward ? order : order + dim_dn;
  const size_t smem = (size_t)dim_dn * (fp64 ? 16 : 8);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e;
  if (fp64) {
    e = cudaFuncSetAttribute(k_permute_cols<double2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_permute_cols<double2><<<dim_up, 256, smem, s>>>(static_cast<const double2*>(src),
                                                      static_cast<double2*>(dst), dim_dn, g);
  } else {
    e = cudaFuncSetAttribute(k_permute_cols<float2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_permute_cols<float2><<<dim_up, 256, smem, s>>>(static_cast<const float2*>(src),
                                                     static_cast<float2*>(dst), dim_dn, g);
  }
  return cudaGetLastError();
}

cudaError_t launch_permute_cols(bool fp64, void* x, int dim_up, int dim_dn, const int32_t* order,
                                bool forward, cudaStream_t s) {
  if (dim_up < 1 || dim_dn < 2) return cudaSuccess;   // nothing to permute
  return permute_cols(fp64, x, x, dim_up, dim_dn, order, forward, s);
}

cudaError_t launch_permute_cols_copy(bool fp64, const void* src, void* dst, int dim_up,
                                     int dim_dn, const int32_t* order, bool forward,
                                     cudaStream_t s) {
  if (dim_up < 1 || dim_dn < 1) return cudaSuccess;   // empty matrix
  if (!src || !dst || !order) return cudaErrorInvalidValue;
  return permute_cols(fp64, src, dst, dim_up, dim_dn, order, forward, s);
}

cudaError_t launch_tridiag_expm(const double* alpha, const double* beta, int n, double tau,
                                double* y, int batch, cudaStream_t s) {
  if (n < 1 || n > kMaxKrylov || batch < 1) return cudaErrorInvalidValue;
  k_tridiag_expm<<<batch, 32, 0, s>>>(alpha, beta, n, tau, y);
  return cudaGetLastError();
}

cudaError_t launch_combine(bool fp64, const BatchArgs& a, int nblk, cudaStream_t s) {
  if (fp64) k_combine<double, true><<<nblk, 256, 0, s>>>(a);
  else k_combine<float, true><<<nblk, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_observe(bool fp64, const BatchArgs& a, int nblk, cudaStream_t s) {
  if (fp64) k_combine<double, false><<<nblk, 256, 0, s>>>(a);
  else k_combine<float, false><<<nblk, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_fermion_op(bool fp64, const void* in, void* out, int dim_up_src,
                              int dim_dn_src, int dim_up_dst, int dim_dn_dst, int spin,
                              const int32_t* map, cudaStream_t s) {
  (void)dim_up_src;
  const int64_t n = (int64_t)dim_up_dst * dim_dn_dst;
  const int g = grid_for(n, 256);
  if (fp64)
    k_fermion_op<double><<<g, 256, 0, s>>>(static_cast<const double2*>(in),
                                           static_cast<double2*>(out), dim_dn_src,
                                           dim_up_dst, dim_dn_dst, spin, map);
  else
    k_fermion_op<float><<<g, 256, 0, s>>>(static_cast<const float2*>(in),
                                          static_cast<float2*>(out), dim_dn_src,
                                          dim_up_dst, dim_dn_dst, spin, map);
  return cudaGetLastError();
}

cudaError_t launch_overlap(bool fp64, const BatchArgs& a, const OverlapArgs& o, int nblk,
                           cudaStream_t s) {
  if (fp64) k_overlap<double><<<nblk, 256, 0, s>>>(a, o);
  else k_overlap<float><<<nblk, 256, 0, s>>>(a, o);
  return cudaGetLastError();
}

cudaError_t launch_transpose(bool fp64, const void* in, void* out, int rows, int cols,
                             cudaStream_t s) {
  const dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  if (fp64)
    k_transpose<double2><<<grid, 256, 0, s>>>(static_cast<const double2*>(in),
                                              static_cast<double2*>(out), rows, cols);
  else
    k_transpose<float2><<<grid, 256, 0, s>>>(static_cast<const float2*>(in),
                                             static_cast<float2*>(out), rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_multidot(const double2* V, int64_t ldV, int k, const double2* w,
                            int64_t D, double2* partial, int nblk, cudaStream_t s) {
  const size_t sm = (size_t)(256 / 32) * k * sizeof(double2);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_multidot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
  }
  k_multidot<<<nblk, 256, sm, s>>>(V, ldV, k, w, D, partial);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cols(const double2* partial, int nblk, int k, double2* out,
                               cudaStream_t s) {
  k_reduce_cols<<<(k + 127) / 128, 128, 0, s>>>(partial, nblk, k, out);
  return cudaGetLastError();
}

cudaError_t launch_multiaxpy(const double2* V, int64_t ldV, int k, const double2* c,
                             double2* w, int64_t D, cudaStream_t s) {
  k_multiaxpy<<<grid_for(D, 256), 256, 0, s>>>(V, ldV, k, c, w, D);
  return cudaGetLastError();
}

cudaError_t launch_combine_real(const double2* V, int64_t ldV, int k, const double* c,
                                double2* y, int64_t D, cudaStream_t s) {
  k_combine_real<<<grid_for(D, 256), 256, 0, s>>>(V, ldV, k, c, y, D);
  return cudaGetLastError();
}

cudaError_t launch_norm_dot(const double2* x, const double2* y, int64_t D, double* partial,
                            int nblk, double* out, cudaStream_t s) {
  k_norm_dot_partial<<<nblk, 256, 0, s>>>(x, y, D, partial);
  k_sum_pairs<<<1, 256, 0, s>>>(partial, nblk, out);
  return cudaGetLastError();
}

cudaError_t launch_scale(double2* x, int64_t D, const double* s_dev, bool inverse_sqrt,
                         cudaStream_t s) {
  k_scale<<<grid_for(D, 256), 256, 0, s>>>(x, D, s_dev, inverse_sqrt ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_axpy_real(double2* y, const double2* x, int64_t D, const double* a_dev,
                             double a_sign, cudaStream_t s) {
  k_axpy_real<<<grid_for(D, 256), 256, 0, s>>>(y, x, D, a_dev, a_sign);
  return cudaGetLastError();
}

cudaError_t launch_random_fill(double2* x, int64_t D, uint64_t seed, cudaStream_t s) {
  k_random_fill<<<grid_for(D, 256), 256, 0, s>>>(x, D, seed);
  return cudaGetLastError();
}

cudaError_t launch_docc_sites(bool fp64, const void* psi, const SectorDev* sec, int dim_up,
                              int dim_dn, int Ns, double* partial, int nblk, double* out,
                              cudaStream_t s) {
  (void)dim_up;
  (void)dim_dn;
  if (fp64)
    k_docc_sites<double><<<nblk, 256, 0, s>>>(static_cast<const double2*>(psi), *sec, Ns,
                                              partial);
  else
    k_docc_sites<float><<<nblk, 256, 0, s>>>(static_cast<const float2*>(psi), *sec, Ns,
                                             partial);
  k_sum_sites<<<1, 32, 0, s>>>(partial, nblk, kMaxSites + 1, out);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* in, bool in_fp64, void* out, bool out_fp64,
                           int64_t n, cudaStream_t s) {
  if (in_fp64 == out_fp64)
    return cudaMemcpyAsync(out, in, n * (in_fp64 ? 16 : 8), cudaMemcpyDeviceToDevice, s);
  if (in_fp64)
    k_convert_c128_c64<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const double2*>(in),
                                                         static_cast<float2*>(out), n);
  else
    k_convert_c64_c128<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const float2*>(in),
                                                         static_cast<double2*>(out), n);
  return cudaGetLastError();
}

}  // namespace ed
