// Stage surrogate inference: the MLP F = L4 o s o L3 o s o L2 o s o L1 o s o L0
// of Sec. 3 (widths 6-128-128-128-128-6, s = GELU in tanh form) applied to
// every particle in place (Sec. 4.3: in-situ inference on device-resident
// particles, with the normalise / de-normalise data preparation fused).
//
// Design (one persistent CTA per SM, three 128-particle tile slots per CTA,
// warp-specialised: 24 epilogue warps, an MMA-issuing warp, a fallback warp):
//  * The weight matrices and bias blocks (BF16, ~117 KB) are copied once per
//    CTA into shared memory by bulk async copies and stay there for all
//    tiles. They are the B operand of every MMA, in the K-major no-swizzle
//    core-matrix layout prepared by the pack kernel.
//  * Each layer's accumulator D[128 particles x N] (FP32) takes 128 columns
//    of tensor memory per slot; the slot's two epilogue warpgroups read it
//    (tcgen05.ld), apply GELU, round to BF16 and write the row back as the A
//    operand of the next layer's MMA. Slots 0 and 1 keep that row in tensor
//    memory (64 columns each, two BF16 per column: tcgen05.st, and the MMA
//    reads A from tensor memory), so their MMAs read only the weights from
//    shared memory and their epilogues touch no shared memory. Tensor memory
//    (512 columns) holds three accumulators but only two activation regions,
//    so slot 2 writes its row to a 32 KB shared-memory buffer in the K-major
//    layout and its MMAs read both operands from shared memory. Three tiles
//    in flight keep the tensor pipe fed while the other slots' epilogues
//    evaluate tanh (measured: 2.42 ms per 2^24 particles, against 2.58 ms
//    with two tensor-memory slots and 2.49 ms with three shared-memory ones).
//  * One lane of the MMA warp issues every MMA with descriptors precomputed
//    once, so a K step costs one add; every hidden-layer MMA is M=128 x
//    N=128 (x K=16). The MMA warp and the warpgroups hand the tensor-memory
//    regions to each other through mbarriers (MMA-complete: commit-arrived;
//    epilogue-complete: 256 thread arrivals).
//  * Biases ride in the MMA: one extra K=16 step multiplies a constant
//    shared-memory A matrix whose first two K columns are 1 by the bias split
//    into BF16 hi and lo parts.
//  * GELU: u = x (c0 + c1 x^2) in packed FP32x2, tanh.approx.f32, and
//    2*GELU = x (1 + tanh u) as an FP32x2 FMA, rounded once to BF16. Hidden
//    activations are stored as 2*GELU(x) and the next layer's weights are
//    pre-scaled by 1/2 (exact in BF16).
//  * Inputs are normalised and outputs de-normalised in double-float
//    arithmetic (FP32 pairs with error-free TwoSum / TwoProd steps), which
//    carries about 44 bits, i.e. FP64-grade constants and rounding, on the
//    FP32 pipes. A slot's next inputs are loaded from HBM while the current
//    tile is in the network.
//  * With a training domain, a particle outside it is not mapped: the
//    epilogue queues it when it reads the input, and a fallback warp of the
//    CTA pushes it through the stage with the plain FP32 pusher
//    (push_f32.cuh) while the tensor pipeline goes on; a full queue spills
//    into a global list for the separate list-mode pusher.
#include "mlp_common.cuh"
#include "push_f32.cuh"

namespace bl {

namespace {

using namespace mlp;

constexpr int SLOTS = 3;
constexpr int TM_SLOTS = 2;                        // slots whose activations stay in tensor memory
constexpr int WG_PER_SLOT = 2;                     // epilogue warpgroups per slot
constexpr int FEAT_WG = 128 / WG_PER_SLOT;         // hidden features per warpgroup
constexpr int CHUNK = 16;                          // accumulator columns per tcgen05.ld
constexpr int EPI_THREADS = 128 * WG_PER_SLOT * SLOTS;
constexpr int EPI_WARPS = EPI_THREADS / 32;
constexpr int THREADS = EPI_THREADS + 64;          // + the MMA warp + the fallback warp
constexpr int MMA_WARP = EPI_WARPS;
constexpr int FB_WARP = EPI_WARPS + 1;
constexpr uint32_t ACT_BYTES = 128 * 128 * 2;      // the shared-memory slot's BF16 activations
constexpr uint32_t OFF_ACT = (MLP_IMG_BYTES + 1023) / 1024 * 1024;
constexpr uint32_t OFF_ONES = OFF_ACT + ACT_BYTES;  // 128 x 16 BF16 A matrix of the bias step
constexpr uint32_t ONES_BYTES = 128 * 16 * 2;
constexpr uint32_t OFF_BAR = OFF_ONES + ONES_BYTES;  // 1 weights + SLOTS mma + SLOTS epi
constexpr uint32_t OFF_SLOT = OFF_BAR + 8 * (1 + 2 * SLOTS);
// fallback queue: indices of this CTA's particles outside the training
// domain (-1 until written), then [0] the queue tail, [1] the number of
// epilogue warps that have finished all their tiles
constexpr int FBQ_CAP = 256;
constexpr uint32_t OFF_FBQ = (OFF_SLOT + 4 + 15) / 16 * 16;
constexpr uint32_t OFF_FBC = OFF_FBQ + FBQ_CAP * 8;
constexpr uint32_t SMEM_BYTES = (OFF_FBC + 8 + 127) / 128 * 128;
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
static_assert(SMEM_BYTES > 114 * 1024, "one CTA per SM (it owns all tensor memory)");
// Tensor memory (columns): slot s's FP32 accumulator at 128 s; the BF16
// activations (the next MMA's A operand, 2 per column) of slots 0 and 1 at
// 384 + 64 s. Slot 2 keeps its activations in shared memory.
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TM_ACC = 128, TM_ACT0 = 384;
static_assert(TM_ACC * SLOTS <= TM_ACT0 && TM_ACT0 + 64 * TM_SLOTS <= TMEM_COLS,
              "tensor memory budget");

// Two hidden pre-activations (FP32 accumulators r0, r1, bias included) ->
// packed BF16 pair of 2*GELU: u = x (c0 + c1 x^2) in FP32x2, tanh.approx.f32,
// x (1 + tanh u) as one FP32x2 FMA, one rounding to BF16 at the end.
BL_DEV uint32_t gelu2_pair(uint32_t r0, uint32_t r1) {
  uint64_t x, x2, p, u, t, y;
  asm("mov.b64 %0, {%1,%2};" : "=l"(x) : "r"(r0), "r"(r1));
  asm("mul.rn.f32x2 %0, %1, %1;" : "=l"(x2) : "l"(x));
  const uint64_t c1 = ((uint64_t)__float_as_uint(GELU_C1) << 32) | __float_as_uint(GELU_C1);
  const uint64_t c0 = ((uint64_t)__float_as_uint(GELU_C0) << 32) | __float_as_uint(GELU_C0);
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(p) : "l"(x2), "l"(c1), "l"(c0));
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(u) : "l"(x), "l"(p));
  uint32_t ulo, uhi, tlo, thi, ylo, yhi, yb;
  asm("mov.b64 {%0,%1}, %2;" : "=r"(ulo), "=r"(uhi) : "l"(u));
  asm("tanh.approx.f32 %0, %1;" : "=r"(tlo) : "r"(ulo));
  asm("tanh.approx.f32 %0, %1;" : "=r"(thi) : "r"(uhi));
  asm("mov.b64 %0, {%1,%2};" : "=l"(t) : "r"(tlo), "r"(thi));
  asm("fma.rn.f32x2 %0, %1, %2, %1;" : "=l"(y) : "l"(x), "l"(t));
  asm("mov.b64 {%0,%1}, %2;" : "=r"(ylo), "=r"(yhi) : "l"(y));
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(yb) : "r"(yhi), "r"(ylo));
  return yb;
}

// GELU of 16 consecutive accumulator columns (features f0 .. f0+15 of each
// of the warp's 32 particle rows), written as 8 columns of packed BF16 pairs
// at activation column f0 / 2 of the warp's lanes (base `t_act`).
BL_DEV void gelu_chunk(const uint32_t (&r)[16], uint32_t t_act, int f0) {
  tc::tmem_st8(t_act + (uint32_t)(f0 / 2), gelu2_pair(r[0], r[1]), gelu2_pair(r[2], r[3]),
               gelu2_pair(r[4], r[5]), gelu2_pair(r[6], r[7]), gelu2_pair(r[8], r[9]),
               gelu2_pair(r[10], r[11]), gelu2_pair(r[12], r[13]), gelu2_pair(r[14], r[15]));
}

// The same 16 columns written as two 16-byte K chunks of the row in the
// shared-memory activation buffer (row base `row`, K chunks 128 bytes apart).
BL_DEV void gelu_chunk_smem(const uint32_t (&r)[16], uint32_t row, int f0) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t a = gelu2_pair(r[8 * q + 0], r[8 * q + 1]);
    const uint32_t b = gelu2_pair(r[8 * q + 2], r[8 * q + 3]);
    const uint32_t d = gelu2_pair(r[8 * q + 4], r[8 * q + 5]);
    const uint32_t e = gelu2_pair(r[8 * q + 6], r[8 * q + 7]);
    tc::st_shared_v4(row + (uint32_t)(f0 / 8 + q) * 128, a, b, d, e);
  }
}

// Epilogue warps of one slot: activations in tensor memory (TM) or in the
// shared-memory buffer (the slot the MMA reads with both operands in shared
// memory).
template <bool TM>
BL_DEV void epilogue(Soa<float> &z, int64_t n, int64_t ntiles, const MlpNormF &nrm,
                     unsigned *err, const MlpDomain &dom, long long *fbq, int *fbc,
                     uint32_t sbase, uint32_t tmem, uint32_t bar_w, int warp, int lane) {
    const int wg = warp >> 2, wq = warp & 3;
    const int slot = wg / WG_PER_SLOT, h = wg % WG_PER_SLOT;
    const bool io = (h == 0);  // this warpgroup loads inputs and stores outputs
    const int m = wq * 32 + lane;  // this thread's particle row within a tile
    const uint32_t t_lane = tmem + ((uint32_t)(wq * 32) << 16);
    const uint32_t t_acc = t_lane + TM_ACC * slot;
    const uint32_t t_act = t_lane + TM_ACT0 + 64 * slot;  // slots in tensor memory
    const uint32_t act = sbase + OFF_ACT;                 // the slot in shared memory
    const uint32_t row_in = act + (uint32_t)((m >> 3) * 256 + (m & 7) * 16);    // K = 16 layout
    const uint32_t row_h = act + (uint32_t)((m >> 3) * 2048 + (m & 7) * 16);    // K = 128 layout
    const uint32_t my_mma = bar_w + 8 * (1 + slot), my_epi = bar_w + 8 * (1 + SLOTS + slot);
    bool ok = __all_sync(0xffffffffu, tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err));
    uint32_t ph = 0;
    auto done = [&]() {  // hand the activations and the accumulator to the MMA warp
      if (TM) tc::tmem_st_wait();
      else tc::fence_proxy_async();
      tc::fence_before();
      mbar_arrive(my_epi);
    };
    auto wait_mma = [&]() {
      ok = ok && __all_sync(0xffffffffu, tc::mbar_wait(my_mma, ph, BL_DEVERR_MMA_TIMEOUT, err));
      ph ^= 1;
      tc::fence_after();
    };
    const int64_t tstride = (int64_t)gridDim.x * SLOTS;
    int64_t tile = (int64_t)blockIdx.x * SLOTS + slot;
    float xin[6];
    {
      const int64_t p = tile * 128 + m;
#pragma unroll
      for (int c = 0; c < 6; ++c) xin[c] = (io && tile < ntiles && p < n) ? z.c[c][p] : 0.0f;
    }
    for (; ok && tile < ntiles; tile += tstride) {
      const int64_t p = tile * 128 + m;
      const bool valid = p < n;
      // outside the training-input box: not mapped, but pushed by the plain
      // pusher (a NaN compares false and is mapped, so it stays visible)
      bool outside = false;
      if (dom.fb_list) {
#pragma unroll
        for (int c = 0; c < 6; ++c) outside |= (xin[c] < dom.lo[c]) | (xin[c] > dom.hi[c]);
        if (io && valid && outside) {
          // to this CTA's fallback warp, or, past its queue, to the global
          // list for the separate list-mode pusher
          const int k = dom.fused ? atomicAdd(&fbc[0], 1) : FBQ_CAP;
          if (k < FBQ_CAP) {
            reinterpret_cast<volatile long long *>(fbq)[k] = p;
          } else {
            const unsigned long long g = atomicAdd(dom.fb_count, 1ull);
            if ((int64_t)g < dom.fb_cap) dom.fb_list[g] = p;
            else outside = false;  // list full (cannot happen with capacity n): keep the map
          }
        }
      }
      if (io) {  // normalised input row (K = 16, see input_row)
        float xn[6];
#pragma unroll
        for (int c = 0; c < 6; ++c)
          xn[c] = df_normalise(xin[c], nrm.mu_in[c][0], nrm.mu_in[c][1], nrm.inv_sd_in[c][0],
                               nrm.inv_sd_in[c][1]);
        uint32_t w[8];
        input_row(xn, w);
        if (TM) {
          tc::tmem_st8(t_act, w[0], w[1], w[2], w[3], w[4], w[5], w[6], w[7]);
        } else {
          tc::st_shared_v4(row_in, w[0], w[1], w[2], w[3]);
          tc::st_shared_v4(row_in + 128, w[4], w[5], w[6], w[7]);
        }
      }
      done();  // layer 0 may start
      if (io) {  // prefetch this slot's next tile while the current one is in the network
        const int64_t tn = tile + tstride, pn = tn * 128 + m;
#pragma unroll
        for (int c = 0; c < 6; ++c) xin[c] = (tn < ntiles && pn < n) ? z.c[c][pn] : 0.0f;
      }
#pragma unroll 1
      for (int l = 0; l < 4; ++l) {
        wait_mma();
        if (!ok) break;
        // this warpgroup's FEAT_WG features in chunks of CHUNK columns; the
        // next chunk's load is in flight while the current one is computed
        const int f_base = h * FEAT_WG;
        uint32_t ra[CHUNK], rb[CHUNK];
        tc::tmem_ld(t_acc + f_base, ra);
        tc::tmem_ld_wait_regs(ra);
#pragma unroll
        for (int c = 0; c < FEAT_WG / CHUNK; c += 2) {
          const int f = f_base + c * CHUNK;
          tc::tmem_ld(t_acc + f + CHUNK, rb);
          if (TM) gelu_chunk(ra, t_act, f);
          else gelu_chunk_smem(ra, row_h, f);
          tc::tmem_ld_wait_regs(rb);
          if (c + 2 < FEAT_WG / CHUNK) tc::tmem_ld(t_acc + f + 2 * CHUNK, ra);
          if (TM) gelu_chunk(rb, t_act, f + CHUNK);
          else gelu_chunk_smem(rb, row_h, f + CHUNK);
          if (c + 2 < FEAT_WG / CHUNK) tc::tmem_ld_wait_regs(ra);
        }
        done();  // layer l+1 may read these activations and overwrite the accumulator
      }
      if (!ok) break;
      wait_mma();  // output layer complete
      if (!ok) break;
      if (!io) continue;
      uint32_t r[8];
      tc::tmem_ld8(t_acc, r);
      tc::tmem_ld_wait();
      if (valid && !outside) {  // particles outside the domain are the pushers'
#pragma unroll
        for (int c = 0; c < 6; ++c)
          z.c[c][p] = df_affine(__uint_as_float(r[c]), nrm.sd_out[c][0], nrm.sd_out[c][1],
                                nrm.mu_out[c][0], nrm.mu_out[c][1]);
      }
    }
    // this warp has queued all its fallback particles
    __syncwarp();
    __threadfence_block();
    if (lane == 0) atomicAdd(&fbc[1], 1);
}

// Registers: the 4 sub-partitions of the SM each hold a quarter of the 64K
// registers, and warp w runs on sub-partition w % 4, so the MMA and fallback
// warps make sub-partitions 0 and 1 host one warp more than the others.
constexpr int WARPS_SMSP0 = (THREADS / 32 + 3) / 4;
constexpr int MAX_REGS = (16384 / (32 * WARPS_SMSP0)) / 8 * 8;

__global__ void __maxnreg__(MAX_REGS)
mlp_forward_kernel(Soa<float> z, int64_t n, int64_t ntiles, const uint8_t *__restrict__ img,
                   MlpNormF nrm, unsigned *err, MlpDomain dom) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint32_t *tslot = reinterpret_cast<uint32_t *>(smem + OFF_SLOT);
  const uint32_t sbase = tc::smem_u32(smem);
  const uint32_t bar_w = sbase + OFF_BAR;
  // mma_done[s] at bar + 8 (1 + s); epi_done[s] at bar + 8 (1 + SLOTS + s)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    tc::mbar_init(bar_w, 1);
    for (int s_ = 0; s_ < SLOTS; ++s_) {
      tc::mbar_init(bar_w + 8 * (1 + s_), 1);
      tc::mbar_init(bar_w + 8 * (1 + SLOTS + s_), 128 * WG_PER_SLOT);
    }
    tc::fence_mbar_init();
  }
  if (warp == MMA_WARP) {
    tc::tmem_alloc(tc::smem_u32(tslot), TMEM_COLS);
    tc::tmem_relinquish();
  }
  long long *fbq = reinterpret_cast<long long *>(smem + OFF_FBQ);
  int *fbc = reinterpret_cast<int *>(smem + OFF_FBC);
  for (int i = tid; i < FBQ_CAP; i += THREADS) fbq[i] = -1;
  if (tid == 0) {
    fbc[0] = 0;
    fbc[1] = 0;
  }
  // constant A operand of the bias step: rows of (1, 1, 0, ..., 0), K-major
  // core matrices (8 rows x 16 bytes, K chunks 128 bytes apart, row groups
  // 256 bytes apart)
  init_ones(smem, OFF_ONES, tid, THREADS);
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0) load_weights(sbase, img, bar_w);

  if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA warp
    // One lane runs the whole issue loop: the 5 layers x SLOTS batches of a
    // tile round are unrolled, so every descriptor is a register plus a
    // compile-time offset and nothing but the epilogue-complete wait stands
    // between two batches.
    if (lane == 0) {
      bool ok = tc::mbar_wait(bar_w, 0, BL_DEVERR_TMA_TIMEOUT, err);
      uint32_t ph = 0;  // bit s: expected phase of epi_done[s]
      constexpr uint32_t ID_H = tc::idesc_bf16(128, 128);
      constexpr uint32_t ID_O = tc::idesc_bf16(128, 16);
      // shared-memory descriptors of the weights; a K step adds 256 bytes (16
      // in the descriptor's address field, which cannot carry for a 228 KB space)
      const uint64_t d_w0 = tc::sdesc(sbase + OFF_W0, 128, 256);
      // layers 1..4: W1, W2, W3, W4 are MLP_IMG_WH bytes apart, and so are the
      // bias blocks B1..B4 at MLP_IMG_BH (the descriptor address is in 16 B units)
      const uint64_t d_w1 = tc::sdesc(sbase + OFF_W1, 128, 2048);
      const uint64_t d_b1 = tc::sdesc(sbase + OFF_B1, 128, 256);
      // A operands: the bias step's constant matrix and slot 2's activations
      // in shared memory (K = 16 layout for the input, K = 128 after); slots
      // 0 and 1 read theirs from tensor memory, 8 columns per K step of 16
      const uint64_t d_ones = tc::sdesc(sbase + OFF_ONES, 128, 256);
      const uint64_t d_in0 = tc::sdesc(sbase + OFF_ACT, 128, 256);
      const uint64_t d_act0 = tc::sdesc(sbase + OFF_ACT, 128, 2048);
      for (int64_t t0 = (int64_t)blockIdx.x * SLOTS; ok && t0 < ntiles;
           t0 += (int64_t)gridDim.x * SLOTS) {
        const int64_t live = ntiles - t0;  // slots s < live hold a tile in this pass
#pragma unroll
        for (int l = 0; l < 5; ++l) {
#pragma unroll
          for (int s_ = 0; s_ < SLOTS; ++s_) {
            if (s_ < live && ok) {
              ok = tc::mbar_wait(bar_w + 8 * (1 + SLOTS + s_), (ph >> s_) & 1u,
                                 BL_DEVERR_MMA_TIMEOUT, err);
              ph ^= 1u << s_;
              if (ok) {
                tc::fence_after();
                const uint32_t acc = tmem + TM_ACC * s_;
                const uint32_t act = tmem + TM_ACT0 + 64 * s_;
                if (l == 0) {
                  if (s_ < TM_SLOTS) tc::mma_ts(acc, act, d_w0, ID_H, 0);
                  else tc::mma_ss(acc, d_in0, d_w0, ID_H, 0);
                } else {
                  const uint64_t dw = d_w1 + (uint64_t)((l - 1) * (MLP_IMG_WH >> 4));
                  const uint64_t db = d_b1 + (uint64_t)((l - 1) * (MLP_IMG_BH >> 4));
                  const uint32_t id = (l < 4) ? ID_H : ID_O;
#pragma unroll
                  for (int j = 0; j < 8; ++j) {
                    if (s_ < TM_SLOTS) tc::mma_ts(acc, act + 8 * j, dw + 16 * j, id, j > 0);
                    else tc::mma_ss(acc, d_act0 + 16 * j, dw + 16 * j, id, j > 0);
                  }
                  tc::mma_ss(acc, d_ones, db, id, 1);
                }
                tc::mma_commit(bar_w + 8 * (1 + s_));
              }
            }
          }
        }
      }
    }
    __syncwarp();
  } else if (warp == FB_WARP) {
    // ------------------------------------------------------- fallback warp
    // Pushes this CTA's particles outside the training domain through the
    // stage with the plain FP32 pusher, 32 at a time (one per lane), while
    // the tensor pipeline goes on with the other tiles. The epilogue queues
    // a particle when it reads the particle's input; the warp leaves once
    // every epilogue warp has finished its tiles and the queue is drained.
    // Every wait is bounded.
    if (dom.fb_list && dom.fused) {
      volatile long long *vq = fbq;
      volatile int *vc = fbc;
      const float4 *table = reinterpret_cast<const float4 *>(dom.table);
      int head = 0;
      uint32_t idle = 0;
      for (;;) {
        int tail = 0, fin = 0;
        if (lane == 0) {
          fin = vc[1];  // read before the tail: a finished warp has queued everything
          tail = min(vc[0], FBQ_CAP);
        }
        tail = __shfl_sync(0xffffffffu, tail, 0);
        fin = __shfl_sync(0xffffffffu, fin, 0);
        if (head < tail) {
          const int k = head + lane;
          if (k < tail) {
            // the entry is written right after its slot is reserved
            long long p = vq[k];
            for (uint32_t w = 0; p < 0 && w < (1u << 22); ++w) p = vq[k];
            if (p >= 0) push::push_particle(z, p, dom.stage, table);
            else atomicOr(err, BL_DEVERR_BARRIER_TIMEOUT);
          }
          __syncwarp();
          head = min(tail, head + 32);
          idle = 0;
          continue;
        }
        if (fin == EPI_WARPS) break;  // nothing queued after the finish count was read
        if (++idle > (1u << 26)) {    // ~30 s of polling: give up and flag it
          if (lane == 0) atomicOr(err, BL_DEVERR_BARRIER_TIMEOUT);
          break;
        }
        __nanosleep(256);
      }
    }
  } else {
    // ------------------------------------------------------ epilogue warps
    const int slot = (warp >> 2) / WG_PER_SLOT;
    if (slot < TM_SLOTS)
      epilogue<true>(z, n, ntiles, nrm, err, dom, fbq, fbc, sbase, tmem, bar_w, warp, lane);
    else
      epilogue<false>(z, n, ntiles, nrm, err, dom, fbq, fbc, sbase, tmem, bar_w, warp, lane);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == MMA_WARP) tc::tmem_dealloc(tmem, TMEM_COLS);
}

__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16 &hi, __nv_bfloat16 &lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

__global__ void mlp_pack_kernel(const float *__restrict__ P, uint8_t *__restrict__ img,
                                float *__restrict__ bias, float *__restrict__ wt,
                                float *__restrict__ wn) {
  const int widths[6] = {6, 128, 128, 128, 128, 6};
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int stride = gridDim.x * blockDim.x;
  __nv_bfloat16 *im = reinterpret_cast<__nv_bfloat16 *>(img);
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  // layer 0: N = 128, K = 16: the weights of the 6 inputs' BF16 high parts
  // (columns 0..5), the bias hi/lo (6, 7), the same weights again for the
  // inputs' low parts (8..13), zeros
  for (int i = tid; i < 128 * 16; i += stride) {
    const int nn = i / 16, k = i % 16;
    __nv_bfloat16 v = zero;
    if (k < 6) v = __float2bfloat16_rn(P[0 + nn * 6 + k]);
    else if (k >= 8 && k < 14) v = __float2bfloat16_rn(P[0 + nn * 6 + (k - 8)]);
    else if (k < 8) {
      __nv_bfloat16 hi, lo;
      split_bf16(P[768 + nn], hi, lo);
      v = (k == 6) ? hi : lo;
    }
    im[img_off(nn, k, 16) / 2] = v;
  }
  // hidden layers 1..3: N = K = 128, weights scaled by 1/2
  const int woff[3] = {896, 17408, 33920};
  const int boff[3] = {17280, 33792, 50304};
  for (int l = 0; l < 3; ++l) {
    __nv_bfloat16 *base = im + (OFF_W1 + l * MLP_IMG_WH) / 2;
    for (int i = tid; i < 128 * 128; i += stride) {
      const int nn = i / 128, k = i % 128;
      base[img_off(nn, k, 128) / 2] = __float2bfloat16_rn(0.5f * P[woff[l] + i]);
    }
    __nv_bfloat16 *bb = im + (OFF_B1 + l * MLP_IMG_BH) / 2;
    for (int i = tid; i < 128 * 16; i += stride) {
      const int nn = i / 16, k = i % 16;
      __nv_bfloat16 v = zero;
      if (k < 2) {
        __nv_bfloat16 hi, lo;
        split_bf16(P[boff[l] + nn], hi, lo);
        v = (k == 0) ? hi : lo;
      }
      bb[img_off(nn, k, 16) / 2] = v;
    }
  }
  // layer 4: N = 16 (6 outputs, zero rows), K = 128, scaled by 1/2; bias block
  {
    __nv_bfloat16 *base = im + OFF_W4 / 2;
    for (int i = tid; i < 16 * 128; i += stride) {
      const int nn = i / 128, k = i % 128;
      const float v = nn < 6 ? 0.5f * P[50432 + nn * 128 + k] : 0.f;
      base[img_off(nn, k, 128) / 2] = __float2bfloat16_rn(v);
    }
    __nv_bfloat16 *bb = im + OFF_B4 / 2;
    for (int i = tid; i < 16 * 16; i += stride) {
      const int nn = i / 16, k = i % 16;
      __nv_bfloat16 v = zero;
      if (nn < 6 && k < 2) {
        __nv_bfloat16 hi, lo;
        split_bf16(P[51200 + nn], hi, lo);
        v = (k == 0) ? hi : lo;
      }
      bb[img_off(nn, k, 16) / 2] = v;
    }
  }
  for (int i = tid; i < MLP_BIAS_FLOATS; i += stride) {
    float v = 0.f;
    if (i < 384) v = P[(i < 128 ? 17280 : (i < 256 ? 33792 : 50304)) + (i & 127)];
    else if (i < 390) v = P[51200 + (i - 384)];
    bias[i] = v;
  }
  // SIMT copies: BF16-rounded weights (unscaled), exact FP32 biases
  for (int l = 0; l < 5; ++l) {
    const int fi = widths[l], fo = widths[l + 1];
    const int wo = (l == 0) ? 0 : (l == 1 ? 896 : (l == 2 ? 17408 : (l == 3 ? 33920 : 50432)));
    const int bo = wo + fi * fo;
    for (int i = tid; i < fi * fo; i += stride) {
      const int o = i / fi, k = i % fi;
      const float w = __bfloat162float(__float2bfloat16_rn(P[wo + i]));
      wn[wo + i] = w;
      wt[wo + k * fo + o] = w;
    }
    for (int i = tid; i < fo; i += stride) {
      wn[bo + i] = P[bo + i];
      wt[bo + i] = P[bo + i];
    }
  }
}

}  // namespace

cudaError_t mlp_forward_configure() {
  return cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)SMEM_BYTES);
}

cudaError_t launch_mlp_pack(const float *params, uint8_t *img, float *bias, float *wt, float *wn,
                            cudaStream_t st) {
  mlp_pack_kernel<<<64, 256, 0, st>>>(params, img, bias, wt, wn);
  return cudaGetLastError();
}

cudaError_t launch_mlp_forward(Soa<float> z, int64_t n, const uint8_t *img, const MlpNorm &nrm64,
                               int num_sms, unsigned *err, cudaStream_t st, const MlpDomain *dom) {
  if (n <= 0) return cudaSuccess;
  const MlpNormF nrm = mlp::norm_pairs(nrm64);
  const int64_t ntiles = (n + 127) / 128;
  int64_t grid = (ntiles + SLOTS - 1) / SLOTS;
  if (grid > num_sms) grid = num_sms;
  MlpDomain d{};
  if (dom) d = *dom;
  mlp_forward_kernel<<<(unsigned)grid, THREADS, SMEM_BYTES, st>>>(z, n, ntiles, img, nrm, err, d);
  return cudaGetLastError();
}

}  // namespace bl
