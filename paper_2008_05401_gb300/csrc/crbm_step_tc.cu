// Tensor-core form of the fused CRBM proposal + Metropolis-Hastings kernel:
// Ising kind, mixed precision, L x L lattices with L = 128 (one chain per CTA),
// 64 (two), 32 (four) or 16 (eight), K <= 4 filters of side k <= 5, mode 0 (S
// proposals of g Gibbs steps).  The chains are the table kernel's chains: the
// same Philox words per unit, and every Bernoulli and MH decision the FP64
// path's.
//
// The three convolutions of a proposal are tcgen05 MMAs with FP32
// accumulators in tensor memory, D[m][n] = sum_kk A[m][kk] B[kk][n] over the
// M = 128 operand rows m:
//   hidden pre-activations of v  (Eq. B2; Eq. 12), one MMA per kernel row a
//       reading the lattice rows i + a;
//   visible pre-activations of h (Eq. B3), per kernel row a the hidden rows
//       i - a, contracted over (filter, hidden column) pairs;
//   hidden pre-activations of v' for F(v') (Eq. 13).
// Operand row m holds lattice row i = m / CH of chain c = m % CH (CH = 128 / L
// chains per CTA, rows interleaved), so that lattice row i + a is operand row
// m + CH a for every chain at once.
// A operands: the 0/1 units in fp16, K-major without swizzle, rows 16 bytes
// apart and 8-column groups one LBO apart, so the operand of kernel row a is
// the same array started CH a rows further on; periodic halos are copies
// (operand rows 128.. repeat rows 0.., the last column group repeats the first;
// hidden planes keep their last rows before row 0).
// B operands: banded Toeplitz images of the filters (built on the host).  Each
// weight is written as W = qf (c2 2^22 + c1 2^11 + c0), qf a power of two and
// integer digits |c| <= 1024 (exact in fp16).  Units times digits summed over
// a window are integers below 2^17, exact in FP32 whatever the order of the
// tensor core's additions, so the only roundings are the quantisation
// (|W - qf W_int| <= qf / 2) and the FP32 combination of the digit sums here.
// Bernoulli decisions use the certified margin of decide32 with this form's
// constants (the FP64 tables decide inside it); the free energy carries its
// error bound into the MH decision like the table kernel's FP32 free energy.
//
// Schedule per Gibbs step: NT = L / 8 hidden tiles of 8 columns (H) and
// NV = L / 16 visible tiles of 16 columns (V), interleaved so that a V tile's
// MMAs run while the epilogue warps work through the two H stages after its
// last input tile (L = 128: H15 H0 H1 H2 H3 V0 H4 H5 V1 ... H12 H13 V5 H14 V6
// V7; L = 32: H3 H0 H1 H2 V0 V1; L = 16: H1 H0 V0); then NT free-energy tiles (F).  Warp-specialised pipeline: two issuing
// warps put each stage's MMAs into one of four tensor-memory buffers and
// commit them to that buffer's `full` mbarrier; the 16 epilogue warps (warp
// w: lanes 32 (w % 4) .. + 31 = operand rows, w / 4 = filter or column
// quarter) take the stages in the same order, read the accumulators, arrive
// on the buffer's `empty` mbarrier and make the stage's decisions.  A V
// stage's MMAs wait on the `hrdy` mbarriers of its three H tiles (every warp's
// fp16 hidden units written and fenced), the F stages on `vrdy` (every warp's
// v' written); CTA barriers only at the end of a proposal (reductions, MH)
// and between Gibbs steps.
#include "crbm_step.cuh"

namespace crbm {
namespace {

constexpr int kEpi = 512, kThr = kEpi + 64;                // 16 epilogue warps + 2 MMA-issuing warps
constexpr int kBhA = 3072;                                 // per kernel row: K=16 x N=96
// visible images, per (kernel row a, K-step j): K=16 x N=48 (1536 B, LBO 768);
// K-step j contracts column groups 2j, 2j+1 of a V buffer's 3K groups
constexpr int kBvStep = 1536;
__host__ __device__ constexpr int v_ksteps(int K) { return (3 * K + 1) / 2; }
constexpr int kTmCols = 512, kTmBuf = 128, kNbuf = 4;

// Geometry of an L x L lattice in the 128-row operands.  A column group holds
// 128 operand rows and HH halo rows: a lattice operand repeats rows 0 .. HH-1
// after row 127 (kernel rows a < 5 read rows m + CH a), a hidden plane of a V
// buffer keeps rows 128-HH .. 127 before row 0 (it is read from row -CH a).
template <int LT>
struct Geo {
  static constexpr int CH = 128 / LT;               // chains per CTA
  static constexpr int NT = LT / 8, NV = LT / 16;    // H / F tiles, V tiles
  static constexpr int GROUPS = LT / 8 + 1;          // operand column groups (the last a halo)
  static constexpr int HH = 4 * CH < 8 ? 8 : 4 * CH; // halo rows (>= CH (k - 1), a multiple of 8)
  static constexpr int ROWS = 128 + HH;
  static constexpr int LBO = ROWS * 16;              // one 8-column group
  static constexpr int PLANE3 = 3 * LBO;             // hidden plane of a V buffer: 3 groups
  static constexpr int VBUF = 4 * PLANE3;
  static constexpr int PGRP = 4 * LBO;               // one column group of 4 hidden planes
  static constexpr int OPV = GROUPS * LBO;
  static constexpr int WPR = LT / 32, WPC = LT * LT / 32;   // words per row / per chain
  static constexpr int NHV = NT + NV;                // H and V stages per Gibbs step
  // misc area: per-chain redo counters at 224 (bytes 0 .. 223 unused), then
  // per (warp, chain) F partials and per-part counts
  static constexpr int REDF = CH <= 4 ? 256 : 288, REDC = REDF + 256 * CH;
  static constexpr int MISC = CH <= 2 ? 1024 : (CH == 4 ? 1536 : 2560);
  static constexpr int SPAN = WPC < 32 ? WPC : 32;   // count-pass lanes per part (one chain's)
  static_assert(LT == 128 || LT == 64 || LT == 32 || LT == 16, "lattice side");
  static_assert(REDC + 64 <= MISC && 224 + 8 * CH <= REDF, "misc area");
};

struct TcLayout {
  uint32_t opv[2], vbuf, plast, hold, bh, bv, vbits, pb[2], hbits, scratch, ch, misc, lut, total;
};

template <int LT>
__host__ __device__ inline TcLayout tc_layout(int K, int k) {
  using G = Geo<LT>;
  TcLayout l;
  uint32_t o = 0;
  l.opv[0] = o; o += G::OPV;          // lattice operands (v; v'), two buffers
  l.opv[1] = o; o += G::OPV;
  l.vbuf = o; o += 2 * G::VBUF;       // hidden operands of V tiles, two buffers of 3 groups
  l.plast = o; o += G::PGRP;          // the last hidden tile, kept for the last V tile
  l.hold = o; o += G::PGRP;           // the last odd hidden tile, until the next even one moves it
  l.bh = o; o += (uint32_t)(k * kBhA);           // filter images: hidden / free energy
  l.bv = o; o += (uint32_t)(k * v_ksteps(K) * kBvStep);   // visible
  l.vbits = o; o += G::CH * G::WPC * 4;         // packed current lattices, chain-major
  l.pb[0] = o; o += G::CH * G::WPC * 4;         // packed proposals (ping-pong over Gibbs steps)
  l.pb[1] = o; o += G::CH * G::WPC * 4;
  l.hbits = o; o += G::CH * 4 * G::WPC * 4;     // packed hidden units: chain, then filter planes
  l.scratch = o; o += 256 * 8;
  l.ch = o; o += (uint32_t)align16(G::CH * sizeof(ChainSm));
  l.misc = o; o += G::MISC;           // mbarriers, TMEM address, counters, reduction slots
  l.lut = o; o += 256 * 16;            // fp16 operand images of the 256 bytes of units
  l.total = o;
  return l;
}

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Instruction descriptor: fp16 x fp16 -> FP32, A and B K-major, M = 128.
__host__ __device__ constexpr uint32_t umma_idesc(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
// High word of every descriptor here: SBO = 128 bytes, version 1.  The low
// word holds the start address and LBO, so operand offsets are 32-bit adds.
constexpr uint32_t kDescHi = (128u >> 4) | (1u << 14);
__device__ __forceinline__ uint32_t umma_desc_lo(uint32_t addr, uint32_t lbo) {
  return ((addr >> 4) & 0x3FFFu) | (((lbo >> 4) & 0x3FFFu) << 16);
}
__device__ __forceinline__ void umma(uint32_t d, uint32_t alo, uint32_t blo, uint32_t id, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\n.reg .b64 da, db;\nsetp.ne.b32 p, %4, 0;\nmov.b64 da, {%1, %5};\n"
               "mov.b64 db, {%2, %5};\ntcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n}\n"
               :: "r"(d), "r"(alo), "r"(blo), "r"(id), "r"(acc), "r"(kDescHi) : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" :: "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tm_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tm_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
// Ties loaded accumulator registers to a point after tm_wait(): volatile asm
// statements keep their order, and every later use of the values now depends
// on this one, so no use can be scheduled before the wait.
__device__ __forceinline__ void tm_tie(float (&v)[4]) {
  asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]));
}
__device__ __forceinline__ void tm_tie(float (&v)[8]) {
  asm volatile("" : "+f"(v[0]), "+f"(v[1]), "+f"(v[2]), "+f"(v[3]), "+f"(v[4]), "+f"(v[5]), "+f"(v[6]), "+f"(v[7]));
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void proxy_fence() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// Wait for the given phase parity of an mbarrier for at most `limit` SM clock
// cycles.  On running out the wait raises the CTA's abort flag (if given) and
// the launch's error flag and returns false; once the abort flag is up every
// wait of the CTA returns false at once, so that the CTA runs to its end
// instead of stalling wait after wait (its results are void and the host
// reports CRBM_ETIMEOUT).  The first probe is inline; the polling loop with its
// clock reads is out of line, so that a phase already complete costs one probe
// and no branch-heavy code at every call site.
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t done;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
               : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
  return done != 0;
}
static __device__ __noinline__ bool mbar_poll(uint32_t mbar, uint32_t parity, long long limit, volatile int* abort,
                                              int* err) {
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(mbar, parity)) return true;
    if (abort != nullptr && *abort != 0) return false;
    if (clock64() - t0 > limit) {
      if (abort != nullptr) *abort = 1;
      if (err != nullptr) atomicExch(err, kErrTimeout);
      return false;
    }
  }
}
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit, volatile int* abort,
                                          int* err) {
  if (mbar_try(mbar, parity)) return true;
  return mbar_poll(mbar, parity, limit, abort, err);
}

// CTA barrier with the tensor-memory and proxy fences around it.
__device__ __forceinline__ void cta_sync() {
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" :: "r"(mbar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" :: "r"(mbar) : "memory");
}
// Arrive from the lanes where `on` holds, as a predicated instruction (no
// branch around it).
__device__ __forceinline__ void mbar_arrive_if(uint32_t mbar, bool on) {
  asm volatile("{\n.reg .pred p;\n.reg .b64 st;\nsetp.ne.u32 p, %1, 0;\n@p mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n"
               :: "r"(mbar), "r"((uint32_t)on) : "memory");
}

enum { kStH = 0, kStV = 1, kStF = 2 };

// Stage z (0 .. NT+NV-1) of a Gibbs step: H_{NT-1} H0 H1 H2 H3, then
// (V_u H_{2u+4} H_{2u+5}) for u = 0 .. NV-4, then V_{NV-3} H_{NT-2} V_{NV-2}
// V_{NV-1}.  V_u reads H tiles 2u-1, 2u, 2u+1 (mod NT); it comes two H stages
// after the last of them, so its MMAs run while the epilogue warps work
// through those stages.
template <int LT>
__device__ __forceinline__ void hv_stage(int z, int& type, int& tile) {
  using G = Geo<LT>;
  if (G::NV == 2) {           // H3 H0 H1 H2 V0 V1
    type = z < 4 ? kStH : kStV;
    tile = z == 0 ? 3 : (z < 4 ? z - 1 : z - 4);
    return;
  }
  if (G::NV == 1) {           // H1 H0 V0
    type = z < 2 ? kStH : kStV;
    tile = z == 0 ? 1 : 0;
    return;
  }
  constexpr int kLoop = 5 + 3 * (G::NV - 3);
  if (z < 5) {
    type = kStH;
    tile = z == 0 ? G::NT - 1 : z - 1;
  } else if (z < kLoop) {
    const int u = (z - 5) / 3, r = (z - 5) - 3 * u;
    type = r == 0 ? kStV : kStH;
    tile = r == 0 ? u : 2 * u + 3 + r;
  } else {
    const int e = z - kLoop;
    type = e == 1 ? kStH : kStV;
    tile = e == 0 ? G::NV - 3 : (e == 1 ? G::NT - 2 : G::NV - 4 + e);
  }
}

// MMAs of one stage into tensor-memory columns dcol, then a commit to mbar,
// by issuer `role` (two issuing threads in different warps share the visible
// stages, whose many small MMAs would otherwise be throttled by the issue
// slots the epilogue warps take; role 1 commits at every stage, so `full`
// counts two arrivals).
// H/F tile t (role 0): N = 96, columns e*32 + f*8 + jj for the digits e = c2,
// c1, c0.  V tile u: N = 48, columns e*16 + jj; the tile's V buffer holds 3K
// column groups (filter f, slot s) at group 3f + s, one LBO apart, so K-step j
// contracts groups 2j, 2j+1 whatever filters they belong to: K-steps j < 3 into
// dcol (role 0), j >= 3 into dcol + 48 (role 1).
// *lo: low descriptor words of the operand bases (start fields advance by byte
// offset / 16).  KT, kT > 0 fix K and k at compile time, so that the issue
// sequence is straight-line code with immediate offsets.
template <int LT, int KT, int kT>
__device__ __forceinline__ void issue_stage(int role, int type, int tile, uint32_t dcol, uint32_t opvlo,
                                            uint32_t vbuflo, uint32_t bhlo, uint32_t bvlo, int Kr, int kr,
                                            uint32_t mbar) {
  using G = Geo<LT>;
  constexpr int CH = G::CH;
  const int K = KT ? KT : Kr, k = kT ? kT : kr;
  if (type != kStV) {
    if (role == 0) {
      const uint32_t id = umma_idesc(96);
      const uint32_t a0 = opvlo + (uint32_t)(tile * (G::LBO >> 4));
#pragma unroll
      for (int a = 0; a < (kT ? kT : 8); ++a)
        if (kT || a < k) umma(dcol, a0 + (uint32_t)(a * CH), bhlo + (uint32_t)(a * (kBhA >> 4)), id, a > 0);
    }
  } else {
    const uint32_t id = umma_idesc(48);
    const uint32_t a0 = vbuflo + (uint32_t)((tile & 1) * (G::VBUF >> 4));
    const int J = v_ksteps(K), j0 = role == 0 ? 0 : 3, j1 = role == 0 ? (J < 3 ? J : 3) : J;
    const uint32_t dc = dcol + (role == 0 ? 0u : 48u);
#pragma unroll
    for (int a = 0; a < (kT ? kT : 8); ++a)
#pragma unroll
      for (int jj = 0; jj < 3; ++jj) {
        const int j = j0 + jj;
        if (j < j1 && (kT || a < k)) {
          const uint32_t aoff = (uint32_t)(2 * j * G::LBO + (G::HH - CH * a) * 16);
          const uint32_t blo = bvlo + (uint32_t)(((a * J + j) * kBvStep) >> 4) + ((768u >> 4) << 16);
          umma(dc, a0 + (aoff >> 4), blo, id, (a | jj) != 0);
        }
      }
  }
  umma_commit(mbar);
}

// FP64 redo of hidden unit (f, n) of a chain from its packed source lattice:
// the FP64 path's sum (h_bias, then kernel rows a = 0..k-1 from the FP64 tables).
template <int LT>
static __device__ __noinline__ uint32_t tc_redo_hidden(const JobDev& jb, int f, const uint32_t* v, int n,
                                                       uint32_t w) {
  const int k = jb.k, T = 1 << k, i = n / LT, j = n - i * LT;
  double x = jb.hb[f];
  for (int a = 0; a < k; ++a) x += __ldg(jb.f64 + (f * k + a) * T + row_window(v, LT, (i + a) % LT, j, k));
  return decide64(x, w);
}

// fp16 units of packed lattices (chain-major) into a lattice operand (ROWS
// rows x GROUPS column groups, the periodic copies included); only the rows of
// chain `only` when only >= 0.
template <int LT>
__device__ void expand_lattice(unsigned char* smem, uint32_t opv, const uint32_t* bits, int tid, int nthr,
                               int only = -1) {
  using G = Geo<LT>;
  const unsigned char* by = (const unsigned char*)bits;
  for (int q = tid; q < G::ROWS * G::GROUPS; q += nthr) {
    const int g = q / G::ROWS, r = q - g * G::ROWS;
    const int rr = r & 127, c = rr % G::CH, i = rr / G::CH;
    if (only >= 0 && c != only) continue;
    const uint32_t x = by[c * (G::WPC * 4) + i * (LT / 8) + (g % G::NT)];
    const uint32_t z = x | (x << 15);       // bit b at b and b + 15: pairs (2p, 2p+1) at 2p and 2p + 16
    uint4 o;
    o.x = ((z >> 0) & 0x10001u) * 0x3C00u;
    o.y = ((z >> 2) & 0x10001u) * 0x3C00u;
    o.z = ((z >> 4) & 0x10001u) * 0x3C00u;
    o.w = ((z >> 6) & 0x10001u) * 0x3C00u;
    *(uint4*)(smem + opv + (uint32_t)g * G::LBO + (uint32_t)r * 16) = o;
  }
}

// The rows of chain c from one lattice operand to another.
template <int LT>
__device__ void copy_chain_rows(unsigned char* smem, uint32_t dst, uint32_t src, int c, int tid, int nthr) {
  using G = Geo<LT>;
  for (int q = tid; q < G::ROWS * G::GROUPS; q += nthr) {
    const int g = q / G::ROWS, r = q - g * G::ROWS;
    if ((r & 127) % G::CH != c) continue;
    const uint32_t off = (uint32_t)g * G::LBO + (uint32_t)r * 16;
    *(uint4*)(smem + dst + off) = *(const uint4*)(smem + src + off);
  }
}

// H tile t, thread (operand row m = lattice row i of its chain), filter f,
// digit sums of its 8 units (f, i, 8t .. 8t+7), Philox words w0, w1: the hidden
// units, packed (into its chain's planes hbc) and as fp16 operands.
template <int LT>
__device__ __forceinline__ void epi_hidden(const JobDev& jb, unsigned char* smem, const TcLayout& ly,
                                           const float (&s2)[8], const float (&s1)[8], const float (&s0)[8],
                                           int m, int i, int f, int t, const uint4& w0, const uint4& w1,
                                           const uint32_t* src, uint32_t hbc, unsigned& nrec) {
  using G = Geo<LT>;
  const int n0 = i * LT + 8 * t;
  const float hb = jb.hb32[f];
  uint32_t byte = 0u, amb = 0u;
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const float x = fmaf(s2[jj], jb.tq2, fmaf(s1[jj], jb.tq1, fmaf(s0[jj], jb.tq0, hb)));
    uint32_t bit, a;
    decide32_split(x, pick(jj < 4 ? w0 : w1, jj & 3), jb.tc0h, jb.tc1, bit, a);
    byte |= bit << jj;
    amb |= a << jj;
  }
  if (amb) {
    // units inside the certified margin: the FP64 path decides (rare)
    for (int jj = 0; jj < 8; ++jj)
      if ((amb >> jj) & 1u) {
        const uint32_t bit = tc_redo_hidden<LT>(jb, f, src, n0 + jj, pick(jj < 4 ? w0 : w1, jj & 3));
        byte = (byte & ~(1u << jj)) | (bit << jj);
        ++nrec;
      }
  }
  smem[hbc + (uint32_t)f * (G::WPC * 4) + (uint32_t)(n0 >> 3)] = (unsigned char)byte;
  const uint4 h4 = *(const uint4*)(smem + ly.lut + byte * 16u);   // the 8 units as fp16 0 / 1
  // operand rows m + HH of the V operands; rows 128-HH..127 also as rows -HH..-1
  const uint32_t r0 = (uint32_t)(m + G::HH) * 16, r1 = (uint32_t)(m - (128 - G::HH)) * 16;
  auto put = [&](uint32_t base) {
    *(uint4*)(smem + base + r0) = h4;
    if (m >= 128 - G::HH) *(uint4*)(smem + base + r1) = h4;
  };
  // V_u reads slots (0, 1, 2) = tiles (2u-1, 2u, 2u+1) of buffer u % 2, last
  // read by V_{u-2}, which precedes H_{2u} in the stage order.  An odd tile goes
  // to the last slot of its V tile and to `hold`; the next (even) H stage moves
  // this thread's rows of it from `hold` to the first slot of the next V tile.
  const int u = t >> 1;
  const uint32_t pf = (uint32_t)f * G::PLANE3, hf = ly.hold + (uint32_t)f * G::LBO;
  if ((t & 1) == 0) {
    const uint32_t vb = ly.vbuf + (uint32_t)(u & 1) * G::VBUF + pf;
    put(vb + 1 * G::LBO);
    *(uint4*)(smem + vb + r0) = *(const uint4*)(smem + hf + r0);
    if (m >= 128 - G::HH) *(uint4*)(smem + vb + r1) = *(const uint4*)(smem + hf + r1);
  } else {
    if (t != G::NT - 1) put(ly.vbuf + (uint32_t)(u & 1) * G::VBUF + pf + 2 * G::LBO);
    else put(ly.plast + (uint32_t)f * G::LBO);   // the last V tile's last slot is in use by earlier V tiles
    put(hf);
  }
}

// V tile u, thread (operand row m = lattice row i of its chain), column
// quarter cq, digit sums of its 4 units (i, 16u + 4cq .. + 3), Philox word w:
// the visible units, packed (into its chain's dbc) and as fp16 F operands.
template <int LT>
__device__ __forceinline__ void epi_visible(const JobDev& jb, unsigned char* smem, const float (&s2)[4],
                                            const float (&s1)[4], const float (&s0)[4], int m, int i, int cq,
                                            int u, const uint4& w, uint32_t* dbc, uint32_t opv,
                                            const uint32_t* hbc, uint32_t hbar, uint32_t parity, long long limit,
                                            volatile int* abort, int* err, unsigned& nrec, uint32_t lut) {
  using G = Geo<LT>;
  const int j0 = 16 * u + 4 * cq, n0 = i * LT + j0;
  uint32_t nib = 0u, amb = 0u;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float x = fmaf(s2[t], jb.tq2, fmaf(s1[t], jb.tq1, fmaf(s0[t], jb.tq0, jb.vb32)));
    uint32_t bit, a;
    decide32_split(x, pick(w, t), jb.tc0v, jb.tc1, bit, a);
    nib |= bit << t;
    amb |= a << t;
  }
  if (amb) {
    // the packed hidden units of H tiles 2u-1, 2u, 2u+1 come from other warps:
    // their hrdy mbarriers (completed before this tile's MMAs) order them
    const int tt[3] = {(2 * u + G::NT - 1) % G::NT, 2 * u, 2 * u + 1};
    for (int q = 0; q < 3; ++q) mbar_wait(hbar + 8u * (uint32_t)tt[q], parity, limit, abort, err);
    for (int t = 0; t < 4; ++t)
      if ((amb >> t) & 1u) {
        const uint32_t bit = recompute_visible(jb, hbc, G::WPC, n0 + t, pick(w, t));
        nib = (nib & ~(1u << t)) | (bit << t);
        ++nrec;
      }
  }
  atomicOr(dbc + (n0 >> 5), nib << (n0 & 31));
  const uint2 h2 = *(const uint2*)(smem + lut + nib * 16u);        // the 4 units as fp16 0 / 1
  const uint32_t off = opv + (uint32_t)(j0 >> 3) * G::LBO + (uint32_t)(j0 & 7) * 2;
  *(uint2*)(smem + off + (uint32_t)m * 16) = h2;
  if (m < G::HH) *(uint2*)(smem + off + (uint32_t)(m + 128) * 16) = h2;
  if (j0 < 8) {        // the last column group repeats the first
    const uint32_t o2 = opv + (uint32_t)G::NT * G::LBO + (uint32_t)(j0 & 7) * 2;
    *(uint2*)(smem + o2 + (uint32_t)m * 16) = h2;
    if (m < G::HH) *(uint2*)(smem + o2 + (uint32_t)(m + 128) * 16) = h2;
  }
}

// F tile, thread (row i, filter f), digit sums of its 8 units: softplus of the
// pre-activations, pairwise sum, Kahan-added into s32 (c32 its compensation).
__device__ __forceinline__ void epi_free(const JobDev& jb, const float (&s2)[8], const float (&s1)[8],
                                         const float (&s0)[8], int f, float& s32, float& c32, float& sabs,
                                         float& ssp) {
  const float hb = jb.hb32[f];
  float sp[8];
#pragma unroll
  for (int jj = 0; jj < 8; ++jj) {
    const float x = fmaf(s2[jj], jb.tq2, fmaf(s1[jj], jb.tq1, fmaf(s0[jj], jb.tq0, hb)));
    sp[jj] = softplus32(x);
    sabs += fabsf(x);
  }
  const float us = ((sp[0] + sp[1]) + (sp[2] + sp[3])) + ((sp[4] + sp[5]) + (sp[6] + sp[7]));
  ssp += us;
  const float y = us - c32;
  const float tt = s32 + y;
  c32 = (tt - s32) - y;
  s32 = tt;
}

// The MH decisions of the chains whose FP32 margin straddled the threshold
// (every thread of the CTA calls; the CH chains' groups of 512 / CH epilogue
// threads work side by side): F of v' with df64 softplus (bound ~1e-7), then
// F of v the same way if only an FP32 value of it is known and the decision
// still straddles; the FP64 path's own code only if that bound still does.
// Out of line, away from the proposal loop's registers.  c0: the chain index
// of the CTA's first chain.
template <int LT>
static __device__ __noinline__ void mh_redo(const JobDev& jb, ChainSm* chs, double* scratch, const uint32_t* pv,
                                            const uint32_t* vbits, uint32_t step, int c0) {
  using G = Geo<LT>;
  const int tid = threadIdx.x, k = jb.k;
  Grp g2;
  g2.tpc = kEpi / G::CH;
  g2.gl = tid / g2.tpc;
  g2.r = tid - g2.gl * g2.tpc;
  const int c = g2.gl < G::CH ? g2.gl : 0;          // this thread's chain (the issuing warps: none)
  ChainSm& ch = chs[c];
  g2.c = c0 + c;
  g2.cid = (uint32_t)(jb.cid_base + (uint64_t)g2.c);
  g2.active = tid < kEpi && ch.flag_rec != 0;
  // the decision with the values known so far: settled (flag_rec 1, flag_acc
  // set) or left to `undecided`
  auto decide = [&](int undecided) {
    const double logr = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
    const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, g2.cid), jb.rk);
    const double logu = log(((double)w.x + 0.5) * 0x1p-32);
    const double Mg = ch.Bp + ch.Fb + ch.lppb + ch.lpb +
                      1e-12 * (fabs(ch.lpp) + fabs(ch.lp) + fabs(ch.Fp) + fabs(ch.F)) + 1e-300;
    ch.flag_rec = 1;
    if (logr - logu > Mg) ch.flag_acc = 1;
    else if (logu - logr > Mg) ch.flag_acc = 0;
    else ch.flag_rec = undecided;
  };
  {
    // F(v') first; F(v), when only its FP32 value is known, only if the
    // decision still straddles (3), since the FP32 bound of F(v) alone is
    // often narrow enough
    double f1[3];
    free_sum_df<4>(jb, g2, pv + c * G::WPC, f1);
    grp_reduce<3>(f1, g2, scratch);
    if (g2.active && g2.r == 0) {
      ch.Fp = -jb.vb * f1[2] - f1[0];
      ch.Bp = f1[1] + 1e-15 * fabs(ch.Fp);
      decide(ch.Fb != 0.0 ? 3 : 2);
      ch.rec_mh += 1ull;
    }
    if (__syncthreads_or(g2.active && g2.r == 0 && ch.flag_rec == 3)) {
      Grp g3 = g2;
      g3.active = g2.active && ch.flag_rec == 3;
      double f2[3];
      free_sum_df<4>(jb, g3, vbits + c * G::WPC, f2);
      grp_reduce<3>(f2, g3, scratch);
      if (g3.active && g3.r == 0) {
        ch.F = -jb.vb * f2[2] - f2[0];
        ch.Fb = f2[1] + 1e-15 * fabs(ch.F);
        decide(2);
      }
    }
  }
  if (__syncthreads_or(g2.active && g2.r == 0 && ch.flag_rec == 2)) {
    Grp g4 = g2;
    g4.active = g2.active && ch.flag_rec == 2;
    Tabs tb64;
    memset(&tb64, 0, sizeof tb64);
    tb64.T = 1 << k;
    tb64.f64 = jb.f64;
    tb64.b64 = jb.b64;
    double f1[4];
    free_energy64(jb, tb64, g4, pv + c * G::WPC, f1);
    grp_reduce<4>(f1, g4, scratch);
    Grp g3 = g4;
    g3.active = g4.active && ch.Fb != 0.0;
    double f2[4];
    free_energy64(jb, tb64, g3, vbits + c * G::WPC, f2);
    grp_reduce<4>(f2, g3, scratch);
    if (g4.active && g4.r == 0) {
      ch.Fp = -jb.vb * f1[2] - f1[0];
      ch.Bp = 0.0;
      if (g3.active) {
        ch.F = -jb.vb * f2[2] - f2[0];
        ch.Fb = 0.0;
      }
      const double logr = (ch.lpp - ch.lp) + (ch.Fp - ch.F);
      const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, g4.cid), jb.rk);
      ch.flag_acc = log(((double)w.x + 0.5) * 0x1p-32) < logr;
    }
  }
}

// mbarriers, in a static shared array (the dynamic layout depends on the
// lattice side of the work item, the barriers' place must not): full[4]
// (count 2, MMA commits), empty[4] (count 16, epilogue warps), hrdy[16]
// (count 16: H tile's fp16 units written), vrdy (count 16: every V tile's v'
// written), fin (count 2, last commits), ld (count 1 plus the byte count of
// the bulk copy of the packed lattices).  Misc area: per-chain Bernoulli redo
// counts at kMiscNrec, then the reduction slots: per (warp, chain) the F
// partial (int64) and its bound (FP32), per warp the lattice counts of the
// chain its count-pass words belong to.
constexpr int kBarFull = 0, kBarEmpty = 4, kBarH = 8, kBarV = 24, kBarFin = 25, kBarLd = 26, kNbar = 27;
constexpr int kMiscNrec = 224;

// Bulk copies between global and shared memory (the TMA unit's untiled form):
// both addresses 16-byte aligned, the size a multiple of 16 bytes.  The load
// completes on an mbarrier that expects its byte count; the store is waited
// for in full (the writes done) before the issuing thread goes on.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" :: "r"(mbar),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
               :: "r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" :: "l"(dst), "r"(src), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
  asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

// One work item of the persistent kernel below: S proposals of the chains
// c0 .. c0 + CH - 1 of job jb (one CTA tile; the last tile of a job may hold
// fewer), the whole pipeline in this CTA's shared memory and in its tensor
// memory at column tmem; bar0: shared address of the CTA's mbarriers (set
// up here, invalidated at the end).  abort: the CTA's abort flag (up once a
// wait has run out; the launch's results are then void).
template <int LT, int KT, int kT, bool EVAL>
__device__ __forceinline__ void tc_tile(const LaunchParams& prm, const JobDev& jb, int c0, unsigned char* smem,
                                        uint32_t bar0, uint32_t tmem, volatile int* abort, uint8_t* stab) {
  using G = Geo<LT>;
  constexpr int CH = G::CH, WPC = G::WPC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool epi = warp < 16;
  const int K = jb.K, k = jb.k;
  const TcLayout ly = tc_layout<LT>(K, k);
  const uint32_t sbase = sm_addr(smem);
  uint32_t* vbits = (uint32_t*)(smem + ly.vbits);
  ChainSm* chs = (ChainSm*)(smem + ly.ch);
  double* scratch = (double*)(smem + ly.scratch);
  auto bar = [&](int b) { return bar0 + 8u * (uint32_t)b; };
  unsigned long long* nrec_sm = (unsigned long long*)(smem + ly.misc + kMiscNrec);
  unsigned char* redf = smem + ly.misc + G::REDF;
  uint32_t* redc = (uint32_t*)(smem + ly.misc + G::REDC);
  auto ch_of = [&](int c) -> ChainSm& { return chs[c]; };
  const int nval = jb.n_chains - c0 < CH ? jb.n_chains - c0 : CH;   // chains of this tile
  const uint32_t vbytes = (uint32_t)(nval * WPC * 4);               // their packed lattices

  // the stage order of a Gibbs step as a table (type | tile << 2), read by
  // the issuing and the epilogue warps at every stage
  if (tid < G::NHV) {
    int ty, tl;
    hv_stage<LT>(tid, ty, tl);
    stab[tid] = (uint8_t)(ty | (tl << 2));
  }
  if (tid == 0) {
    for (int b = 0; b < kNbuf; ++b) {
      mbar_init(bar(kBarFull + b), 2);
      mbar_init(bar(kBarEmpty + b), 16);
    }
    for (int t = 0; t < 16; ++t) mbar_init(bar(kBarH + t), 16);
    mbar_init(bar(kBarV), 16);
    mbar_init(bar(kBarFin), 2);
    mbar_init(bar(kBarLd), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    // the tile's packed lattices (chain-major, contiguous in the job) by one
    // bulk copy: offsets and sizes are multiples of 32 bytes
    mbar_expect_tx(bar(kBarLd), vbytes);
    bulk_load(sbase + ly.vbits, jb.bits + (size_t)c0 * WPC, vbytes, bar(kBarLd));
  }
  const int nimg = (k * kBhA + k * v_ksteps(K) * kBvStep) / 16;   // B images: hidden/free, then visible
  for (int q = tid; q < nimg; q += kThr) ((uint4*)(smem + ly.bh))[q] = __ldg(jb.tcw + q);
  // V buffers zeroed: the groups of filters f >= K are read (with zero weights)
  // by the last K-step when 3K is odd, and must hold finite values
  for (int q = tid; q < 2 * G::VBUF / 16; q += kThr) ((uint4*)(smem + ly.vbuf))[q] = make_uint4(0u, 0u, 0u, 0u);
  for (int q = tid; q < 256; q += kThr) {
    const uint32_t z = (uint32_t)q | ((uint32_t)q << 15);   // bit b at b and b + 15: pairs (2p, 2p+1) at 2p and 2p + 16
    ((uint4*)(smem + ly.lut))[q] = make_uint4(((z >> 0) & 0x10001u) * 0x3C00u, ((z >> 2) & 0x10001u) * 0x3C00u,
                                              ((z >> 4) & 0x10001u) * 0x3C00u, ((z >> 6) & 0x10001u) * 0x3C00u);
  }
  for (int w = tid; w < CH * WPC; w += kThr) {
    if (w >= nval * WPC) vbits[w] = 0u;       // empty chain slots of a short last tile
    ((uint32_t*)(smem + ly.pb[0]))[w] = 0u;
    ((uint32_t*)(smem + ly.pb[1]))[w] = 0u;
  }
  if (tid < CH) {
    ChainSm& ch = ch_of(tid);
    const int c = c0 + tid;
    const bool on = tid < nval;
    ch.F = on ? jb.F[c] : 0.0;
    ch.Fb = on ? jb.Fb[c] : 0.0;
    ch.lpb = on ? jb.Lb[c] : 0.0;
    ch.lppb = 0.0;
    ch.lp = on ? jb.logpi[c] : 0.0;
    ch.E = on ? jb.Ephys[c] : 0.0;
    for (int o = 0; o < kNobs; ++o) {
      ch.ot[o] = on ? jb.obs_t[(size_t)c * kNobs + o] : 0.0;
      ch.os[o] = on ? jb.obs[(size_t)c * kNobs + o] : 0.0;
    }
    ch.beta = on ? 1.0 / jb.T[c] : 1.0;
    // margin terms that do not depend on the proposal: the tile's constants
    // (the fixed-point conversion rounds each thread's sum by <= 2^-33) and
    // those of the current state, renewed whenever the state changes
    ch.cst = (double)K * (double)(LT * LT) * ((double)jb.csp + (double)jb.tcft) + (double)(kEpi / CH) * 0x1p-33;
    ch.mgs = ((ch.Fb + ch.lpb) + 1e-12 * (fabs(ch.lp) + fabs(ch.F))) + (ch.cst + 1e-300);
    ch.acc = 0ull;
    ch.rec_mh = 0ull;
    ch.flag_rec = 0;
    ch.flag_acc = 0;
    nrec_sm[tid] = 0ull;
  }
  // the bulk copy is waited for whatever the abort flag says: it completes by itself
  mbar_wait(bar(kBarLd), 0u, prm.wait_limit, nullptr, prm.err);
  __syncthreads();
  expand_lattice<LT>(smem, ly.opv[0], vbits, tid, kThr);
  cta_sync();

  // epilogue thread: operand row m = lattice row i of chain cm; filter /
  // column quarter fq; its TMEM lanes
  const int m = 32 * (warp & 3) + lane, fq = warp >> 2, i = m / CH, cm = m % CH;
  const uint32_t cid = (uint32_t)(jb.cid_base + (uint64_t)(c0 + cm));
  const uint32_t tlane = (uint32_t)(32 * (warp & 3)) << 16;
  uint32_t* vb_m = vbits + cm * WPC;                           // this thread's chain's planes
  const uint32_t hbc = ly.hbits + (uint32_t)cm * (4 * WPC * 4);
  const bool issuer = warp >= 16 && lane == 0;
  const int role = warp - 16;                     // issuers: 0 and 1

  const uint32_t dopv0 = umma_desc_lo(sbase + ly.opv[0], G::LBO);   // operand x at + x OPV / 16
  const uint32_t dvbuf = umma_desc_lo(sbase + ly.vbuf, G::LBO), dbh = umma_desc_lo(sbase + ly.bh, 1536),
                 dbv = umma_desc_lo(sbase + ly.bv, 0);     // LBO set per image
  uint32_t zc = 0;              // stages so far: buffer zc % 4, its (zc / 4)-th use
  uint32_t gs = 0;              // Gibbs steps so far: phase of hrdy / vrdy
  unsigned nrec = 0;
  const unsigned long long step0 = *(volatile unsigned long long*)jb.step;
  auto wait_bar = [&](uint32_t b, uint32_t parity) { mbar_wait(b, parity, prm.wait_limit, abort, prm.err); };
  // issuing warp: before the MMAs of stage zc, its buffer's previous use read by every epilogue warp
  auto mma_claim = [&]() {
    const uint32_t b = zc & (kNbuf - 1), use = zc / kNbuf;
    if (use > 0) wait_bar(bar(kBarEmpty + b), (use - 1) & 1u);
    tc_fence_after();
    return tmem + b * kTmBuf;
  };
  // epilogue warp: the MMAs of stage zc are done
  auto epi_claim = [&]() {
    const uint32_t b = zc & (kNbuf - 1), use = zc / kNbuf;
    wait_bar(bar(kBarFull + b), use & 1u);
    tc_fence_after();
    return tmem + tlane + b * kTmBuf;
  };
  // epilogue warp: accumulators of stage zc read
  auto epi_release = [&]() {
    tc_fence_before();
    __syncwarp();
    mbar_arrive_if(bar(kBarEmpty + (zc & (kNbuf - 1))), lane == 0);
  };
  // epilogue warp: its generic-proxy operand writes visible to later MMAs, then arrive
  auto epi_publish = [&](uint32_t b) {
    proxy_fence();
    __syncwarp();
    mbar_arrive_if(b, lane == 0);
  };

  if constexpr (EVAL) {
    // evaluation of the current lattices (the values a mixed proposal leaves
    // for an accepted state): the F tiles on operand 0 (v) with the certified
    // FP32 bound, the lattice counts, then F, its bound, log pi = -beta E and
    // the observables; sums, accepts and the step counter are untouched
    float s32 = 0.f, c32 = 0.f, sabs = 0.f, ssp = 0.f;
    if (issuer) {
      for (int t = 0; t < G::NT; ++t, ++zc) {
        const uint32_t d = mma_claim();
        issue_stage<LT, KT, kT>(role, kStF, t, d, dopv0, dvbuf, dbh, dbv, K, k, bar(kBarFull + (zc & (kNbuf - 1))));
      }
    } else if (epi) {
      for (int t = 0; t < G::NT; ++t, ++zc) {
        const uint32_t tcol = epi_claim();
        if (fq < K) {
          float s2[8], s1[8], s0[8];
          tm_ld8(tcol + 8 * fq, s2);
          tm_ld8(tcol + 32 + 8 * fq, s1);
          tm_ld8(tcol + 64 + 8 * fq, s0);
          tm_wait();
          tm_tie(s2);
          tm_tie(s1);
          tm_tie(s0);
          epi_release();
          epi_free(jb, s2, s1, s0, fq, s32, c32, sabs, ssp);
        } else {
          epi_release();
        }
      }
    }
    if (epi) {
      long long fs = __float2ll_rn(s32 * 0x1p32f);
      float bnd = sabs * 0x1p-23f + ssp * (8.0f * 0x1p-24f);
#pragma unroll
      for (int o = 16; o >= CH; o >>= 1) {
        fs += __shfl_xor_sync(kFull, fs, o);
        bnd += __shfl_xor_sync(kFull, bnd, o);
      }
      if (lane < CH) {
        *(long long*)(redf + 16 * (warp * CH + lane)) = fs;
        *(float*)(redf + 16 * (warp * CH + lane) + 8) = bnd;
      }
      uint32_t cnt = 0;
      if (tid < CH * WPC) {
        const uint32_t* p = vbits + (tid / WPC) * WPC;
        const int w = tid % WPC;
        const uint32_t x = p[w];
        uint32_t right, down;
        if constexpr (LT >= 32) {
          const uint32_t xr = p[(w & ~(G::WPR - 1)) | ((w + 1) & (G::WPR - 1))];
          right = (x >> 1) | (xr << 31);
          down = p[(w + G::WPR) % WPC];
        } else {
          right = ((x >> 1) & 0x7FFF7FFFu) | ((x << 15) & 0x80008000u);
          down = (x >> 16) | (p[(w + 1) % WPC] << 16);
        }
        cnt = (uint32_t)__popc(x) | ((uint32_t)(__popc(x ^ right) + __popc(x ^ down)) << 16);
      }
#pragma unroll
      for (int o = G::SPAN / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
      if (tid % G::SPAN == 0 && tid < 16 * G::SPAN) redc[tid / G::SPAN] = cnt;
    }
    __syncthreads();
    if (tid < CH) {
      ChainSm& ch = ch_of(tid);
      long long fs = 0;
      float bnd = 0.0f;
      uint32_t ones = 0, pairs = 0;
      for (int w = 0; w < 16; ++w) {
        fs += *(const long long*)(redf + 16 * (w * CH + tid));
        bnd += *(const float*)(redf + 16 * (w * CH + tid) + 8);
      }
      for (int w = 0; w < 16; ++w)
        if (w * G::SPAN < CH * WPC && (w * G::SPAN) / WPC == tid) {
          ones += redc[w] & 0xFFFFu;
          pairs += redc[w] >> 16;
        }
      constexpr int kN = LT * LT;
      const double Fdata = (double)bnd * 1.001;
      const double E = -jb.J[0] * (double)(2 * kN - 2 * (int)pairs);
      const double M = (double)(2 * (int)ones - kN);
      const double Fv = fma((double)fs, -0x1p-32, -jb.vb * (double)ones);
      ch.F = Fv;
      ch.Fb = (Fdata + ch.cst) + 1e-12 * fabs(Fv);
      ch.lp = -ch.beta * E;
      ch.lpb = 0.0;
      ch.E = E;
      ch.ot[0] = E; ch.ot[1] = E * E; ch.ot[2] = fabs(M); ch.ot[3] = M * M;
    }
  } else {
    for (int s = 0; s < prm.S; ++s) {
      const uint32_t step = (uint32_t)(step0 + (uint64_t)s);
      if (warp == 17 && lane >= 1 && lane <= CH && prm.correct) {
        // the MH draws of this proposal, ahead of the decisions (read after the
        // barriers of the proposal's end).  In FP32, within 2^-20 (1 + |log u|)
        // of the FP64 log u, which the decision adds to its margin: the FP64 log
        // would hold this warp's issuing lane, whose commits every stage waits
        // for, for thousands of cycles on the 1/64-rate FP64 pipe
        const uint4 w = philox4x32_10_rk(make_uint4(0u, kTagAcc, step, (uint32_t)(jb.cid_base + (uint64_t)(c0 + lane - 1))),
                                         jb.rk);
        ch_of(lane - 1).logu = (double)log_u32(w.x);
      }
      // Gibbs step sub reads operand sub % 2 and writes the other: v is in
      // operand 0 at the start of a proposal, v' in operand g % 2 at its end
      for (int sub = 0; sub < prm.g; ++sub, ++gs) {
        const int src = sub & 1;
        const uint32_t pbs = ly.pb[0] + (uint32_t)(sub & 1) * (CH * WPC * 4);
        uint32_t* dbc = (uint32_t*)(smem + pbs) + cm * WPC;
        const uint32_t* sbc =
            sub == 0 ? vb_m : (const uint32_t*)(smem + ly.pb[0] + (uint32_t)((sub - 1) & 1) * (CH * WPC * 4)) + cm * WPC;
        const uint32_t taghid = (uint32_t)(sub * (K + 1)), tagvis = (uint32_t)(sub * (K + 1) + K);
        const uint32_t opv_dst = ly.opv[0] + (uint32_t)(src ^ 1) * G::OPV;
        const uint32_t zbase = zc;
        if (issuer) {
          for (int z = 0; z < G::NHV; ++z, ++zc) {
            const int ty = stab[z] & 3, tl = stab[z] >> 2;
            const uint32_t d = mma_claim();
            if (ty == kStV) {
              wait_bar(bar(kBarH + ((2 * tl + G::NT - 1) % G::NT)), gs & 1u);
              wait_bar(bar(kBarH + 2 * tl), gs & 1u);
              wait_bar(bar(kBarH + 2 * tl + 1), gs & 1u);
              tc_fence_after();
            }
            issue_stage<LT, KT, kT>(role, ty, tl, d, dopv0 + (uint32_t)(src * (G::OPV >> 4)), dvbuf, dbh, dbv, K,
                                    k, bar(kBarFull + (zc & (kNbuf - 1))));
          }
        } else if (epi) {
          for (int z = 0; z < G::NHV; ++z, ++zc) {
            const int ty = stab[z] & 3, tl = stab[z] >> 2;
            // this stage's Philox words do not depend on its MMAs: drawn before
            // waiting for them, so the counter-based generator overlaps the
            // tensor-core work and the accumulator loads
            uint4 w0 = make_uint4(0u, 0u, 0u, 0u), w1 = w0;
            if (ty == kStH) {
              if (fq < K) {
                const uint32_t q0 = (uint32_t)((i * LT + 8 * tl) >> 2), tag = taghid + (uint32_t)fq;
                w0 = philox4x32_10_rk(make_uint4(q0, tag, step, cid), jb.rk);
                w1 = philox4x32_10_rk(make_uint4(q0 + 1u, tag, step, cid), jb.rk);
              }
            } else {
              w0 = philox4x32_10_rk(make_uint4((uint32_t)((i * LT + 16 * tl + 4 * fq) >> 2), tagvis, step, cid),
                                    jb.rk);
              w1 = w0;
            }
            const uint32_t tcol = epi_claim();
            if (ty == kStH) {
              if (fq < K) {
                float s2[8], s1[8], s0[8];
                tm_ld8(tcol + 8 * fq, s2);
                tm_ld8(tcol + 32 + 8 * fq, s1);
                tm_ld8(tcol + 64 + 8 * fq, s0);
                tm_wait();
                tm_tie(s2);
                tm_tie(s1);
                tm_tie(s0);
                epi_release();
                epi_hidden<LT>(jb, smem, ly, s2, s1, s0, m, i, fq, tl, w0, w1, sbc, hbc, nrec);
              } else {
                epi_release();
              }
              if (tl == G::NT - 2 && fq < K) {
                // this thread's rows of the last hidden tile (written by it at the
                // first H stage) into the last slot of the last V tile's buffer,
                // read last by V_{NV-3}, whose MMAs this warp has waited for
                const uint32_t dst = ly.vbuf + (uint32_t)((G::NV - 1) & 1) * G::VBUF + (uint32_t)fq * G::PLANE3 +
                                     2 * G::LBO,
                               pl = ly.plast + (uint32_t)fq * G::LBO;
                const uint32_t r0 = (uint32_t)(m + G::HH) * 16, r1 = (uint32_t)(m - (128 - G::HH)) * 16;
                *(uint4*)(smem + dst + r0) = *(const uint4*)(smem + pl + r0);
                if (m >= 128 - G::HH) *(uint4*)(smem + dst + r1) = *(const uint4*)(smem + pl + r1);
              }
              epi_publish(bar(kBarH + tl));
            } else {
              float s2[4], s1[4], s0[4];
              tm_ld4(tcol + 4 * fq, s2);
              tm_ld4(tcol + 16 + 4 * fq, s1);
              tm_ld4(tcol + 32 + 4 * fq, s0);
              if (K > 2) {
                // K-steps 3.. from the second issuer's accumulator (integer sums: exact)
                float t2[4], t1[4], t0[4];
                tm_ld4(tcol + 48 + 4 * fq, t2);
                tm_ld4(tcol + 64 + 4 * fq, t1);
                tm_ld4(tcol + 80 + 4 * fq, t0);
                tm_wait();
                tm_tie(s2);
                tm_tie(s1);
                tm_tie(s0);
                tm_tie(t2);
                tm_tie(t1);
                tm_tie(t0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  s2[q] += t2[q];
                  s1[q] += t1[q];
                  s0[q] += t0[q];
                }
              } else {
                tm_wait();
                tm_tie(s2);
                tm_tie(s1);
                tm_tie(s0);
              }
              epi_release();
              epi_visible<LT>(jb, smem, s2, s1, s0, m, i, fq, tl, w0, dbc, opv_dst,
                              (const uint32_t*)(smem + hbc), bar(kBarH), gs & 1u, prm.wait_limit, abort,
                              prm.err, nrec, ly.lut);
              if (tl == G::NV - 1) epi_publish(bar(kBarV));
            }
          }
        }
        zc = zbase + G::NHV;
        if (sub + 1 < prm.g) {
          // next Gibbs step: its source is this step's v' (every write done), and
          // the proposal buffer it fills is cleared
          cta_sync();
          for (int w = tid; w < CH * WPC; w += kThr)
            ((uint32_t*)(smem + ly.pb[0] + (uint32_t)((sub + 1) & 1) * (CH * WPC * 4)))[w] = 0u;
          __syncthreads();
        }
      }
      const int fin = prm.g & 1;                                     // operand holding v'
      const uint32_t* pv = (const uint32_t*)(smem + ly.pb[0] + (uint32_t)((prm.g - 1) & 1) * (CH * WPC * 4));

      // free energy of v' from the F tiles
      float s32 = 0.f, c32 = 0.f, sabs = 0.f, ssp = 0.f;
      const uint32_t zbase = zc;
      if (issuer) {
        for (int t = 0; t < G::NT; ++t, ++zc) {
          const uint32_t d = mma_claim();
          if (t == 0) {
            wait_bar(bar(kBarV), (gs - 1) & 1u);
            tc_fence_after();
          }
          issue_stage<LT, KT, kT>(role, kStF, t, d, dopv0 + (uint32_t)(fin * (G::OPV >> 4)), dvbuf, dbh, dbv, K, k,
                                  bar(kBarFull + (zc & (kNbuf - 1))));
        }
      } else if (epi) {
        for (int t = 0; t < G::NT; ++t, ++zc) {
          const uint32_t tcol = epi_claim();
          if (fq < K) {
            float s2[8], s1[8], s0[8];
            tm_ld8(tcol + 8 * fq, s2);
            tm_ld8(tcol + 32 + 8 * fq, s1);
            tm_ld8(tcol + 64 + 8 * fq, s0);
            tm_wait();
            tm_tie(s2);
            tm_tie(s1);
            tm_tie(s0);
            epi_release();
            epi_free(jb, s2, s1, s0, fq, s32, c32, sabs, ssp);
          } else {
            epi_release();
          }
        }
      }
      zc = zbase + G::NT;

      // per-warp sums: F as an exact 2^-32 fixed-point integer and its
      // error-bound part in FP32 per chain (a thread's units are all of its
      // chain cm: lane parity for CH = 2), ones and unequal nearest-neighbour
      // pairs of the count-pass words (every warp's v' writes done: vrdy,
      // completed before the F stages)
      if (epi) {
        wait_bar(bar(kBarV), (gs - 1) & 1u);
        long long fs = __float2ll_rn(s32 * 0x1p32f);
        float bnd = sabs * 0x1p-23f + ssp * (8.0f * 0x1p-24f);
#pragma unroll
        for (int o = 16; o >= CH; o >>= 1) {
          fs += __shfl_xor_sync(kFull, fs, o);
          bnd += __shfl_xor_sync(kFull, bnd, o);
        }
        if (lane < CH) {
          *(long long*)(redf + 16 * (warp * CH + lane)) = fs;
          *(float*)(redf + 16 * (warp * CH + lane) + 8) = bnd;
        }
        uint32_t cnt = 0;
        if (tid < CH * WPC) {
          const uint32_t* p = pv + (tid / WPC) * WPC;
          const int w = tid % WPC;
          const uint32_t x = p[w];
          uint32_t right, down;
          if constexpr (LT >= 32) {          // whole rows of WPR words
            const uint32_t xr = p[(w & ~(G::WPR - 1)) | ((w + 1) & (G::WPR - 1))];
            right = (x >> 1) | (xr << 31);
            down = p[(w + G::WPR) % WPC];
          } else {                           // L = 16: two rows per word
            right = ((x >> 1) & 0x7FFF7FFFu) | ((x << 15) & 0x80008000u);
            down = (x >> 16) | (p[(w + 1) % WPC] << 16);
          }
          cnt = (uint32_t)__popc(x) | ((uint32_t)(__popc(x ^ right) + __popc(x ^ down)) << 16);
        }
#pragma unroll
        for (int o = G::SPAN / 2; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if (tid % G::SPAN == 0 && tid < 16 * G::SPAN) redc[tid / G::SPAN] = cnt;   // part = chain's words
      }
      __syncthreads();
      // thread c < CH: the MH decision of chain c0 + c
      // after the decision, by a lane of warp 1 per chain (beside the accept
      // copies): the accepted state, its observables, the running sums and
      // the state's margin terms for the next decision
      auto settle = [&](ChainSm& ch, int c) {
        if (ch.flag_acc) {
          ch.F = ch.Fp;
          ch.Fb = ch.Bp;
          ch.lp = ch.lpp;
          ch.lpb = ch.lppb;
          ch.E = ch.Ep;
          const double M = (double)(2 * ch.onesp - LT * LT);
          ch.ot[0] = ch.Ep;
          ch.ot[1] = ch.Ep * ch.Ep;
          ch.ot[2] = fabs(M);
          ch.ot[3] = M * M;
          ch.acc += 1ull;
        }
        // (a second-level recompute may also have tightened F(v) of a rejected proposal)
        ch.mgs = ((ch.Fb + ch.lpb) + 1e-12 * (fabs(ch.lp) + fabs(ch.F))) + (ch.cst + 1e-300);
        for (int o = 0; o < kNobs; ++o) ch.os[o] += ch.ot[o];
        if (c0 + c < jb.n_chains) trace_store(jb, c0 + c, step0 + (uint64_t)s, ch.E);
      };
      if (tid < CH) {
        // one thread per chain; each FP64 instruction (conversions included)
        // holds the SMSP's slow FP64 pipe for tens of cycles, so FP64 work is
        // kept small: partial sums in integers and FP32, values in registers
        ChainSm& ch = ch_of(tid);
        const double lp = ch.lp, F = ch.F, Fb = ch.Fb, lpb = ch.lpb, beta = ch.beta, logu = ch.logu;
        long long fs = 0;
        float bnd = 0.0f;
        uint32_t ones = 0, pairs = 0;
        for (int w = 0; w < 16; ++w) {
          fs += *(const long long*)(redf + 16 * (w * CH + tid));
          bnd += *(const float*)(redf + 16 * (w * CH + tid) + 8);
        }
        for (int w = 0; w < 16; ++w)
          if (w * G::SPAN < CH * WPC && (w * G::SPAN) / WPC == tid) {
            ones += redc[w] & 0xFFFFu;
            pairs += redc[w] >> 16;
          }
        // the FP32 sums of the non-negative bound terms over 512 / CH threads and
        // then over 16 warps lose < 26 2^-24 relative, inside the factor 1.001
        constexpr int kN = LT * LT;
        // the margin terms known before this proposal's sums come precomputed
        // (ch.cst, ch.mgs); the observables wait for the decision
        const double cst = ch.cst, mg0 = ch.mgs;
        const double Fdata = (double)bnd * 1.001;
        const double E = -jb.J[0] * (double)(2 * kN - 2 * (int)pairs);
        const double lpp = -beta * E;
        const double Fp = fma((double)fs, -0x1p-32, -jb.vb * (double)ones);
        const double Bp = (Fdata + cst) + 1e-12 * fabs(Fp);
        ch.Ep = E;
        ch.lpp = lpp;
        ch.onesp = (int)ones;
        ch.lppb = 0.0;
        ch.Fp = Fp;
        ch.Bp = Bp;
        ch.flag_rec = 0;
        if (!prm.correct) {
          ch.flag_acc = 1;
        } else {
          const double logr = (lpp - lp) + (Fp - F);
          // = Bp + Fb + lpb + 1e-12 (|lpp| + |lp| + |Fp| + |F|) + 1e-300
          const double Mg = (Fdata + mg0) + 1e-12 * (2.0 * fabs(Fp) + fabs(lpp)) + 0x1p-20 * (1.0 + fabs(logu));
          if (logr - logu > Mg) ch.flag_acc = 1;
          else if (logu - logr > Mg) ch.flag_acc = 0;
          else ch.flag_rec = 1;
        }
      }
      if (__syncthreads_or(tid < CH && ch_of(tid).flag_rec)) {
        mh_redo<LT>(jb, &ch_of(0), scratch, pv, vbits, step, c0);
        __syncthreads();
      }
      if (warp == 1 && lane < CH) settle(ch_of(lane), lane);
      // accepted: v' becomes v (packed, and its operand rows into operand 0 when
      // they are in operand 1); rejected after several Gibbs steps: operand 0
      // was overwritten, so v is expanded again
      for (int c = 0; c < CH; ++c) {
        const bool acc = ch_of(c).flag_acc != 0;
        for (int w = tid; w < WPC; w += kThr) {
          uint32_t* pvw = (uint32_t*)pv + c * WPC;
          if (acc) vbits[c * WPC + w] = pvw[w];
          pvw[w] = 0u;                              // cleared for the next proposal
        }
        if (acc && fin == 1) copy_chain_rows<LT>(smem, ly.opv[0], ly.opv[1], c, tid, kThr);
      }
      __syncthreads();
      for (int c = 0; c < CH; ++c)
        if (!ch_of(c).flag_acc && prm.g > 1) expand_lattice<LT>(smem, ly.opv[0], vbits, tid, kThr, c);
      cta_sync();
    }
  }

  if (nrec) atomicAdd(nrec_sm + cm, (unsigned long long)nrec);
  // every MMA of the item has completed before the next item (or the end of
  // the kernel) reuses shared and tensor memory: the issuers' last commit,
  // waited for whatever the abort flag says (issued MMAs always finish)
  if (issuer) {
    umma_commit(bar(kBarFin));
    mbar_wait(bar(kBarFin), 0u, prm.wait_limit, nullptr, prm.err);
  }
  cta_sync();      // with the proxy fence: the packed lattices visible to the bulk copy
  if (tid == 0) bulk_store(jb.bits + (size_t)c0 * WPC, sbase + ly.vbits, vbytes);
  if (tid < nval) {
    const ChainSm& ch = ch_of(tid);
    const int c = c0 + tid;
    jb.F[c] = ch.F;
    jb.Fb[c] = ch.Fb;
    jb.Lb[c] = ch.lpb;
    jb.logpi[c] = ch.lp;
    jb.Ephys[c] = ch.E;
    for (int o = 0; o < kNobs; ++o) {
      jb.obs_t[(size_t)c * kNobs + o] = ch.ot[o];
      jb.obs[(size_t)c * kNobs + o] = ch.os[o];
    }
    jb.acc[c] += ch.acc;
    jb.rec[2 * (size_t)c] += nrec_sm[tid];
    jb.rec[2 * (size_t)c + 1] += ch.rec_mh;
  }
  if (tid == 0)        // no wait or arrival is pending: the next item initialises them afresh
    for (int b = 0; b < kNbar; ++b) asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" :: "r"(bar(b)) : "memory");
  __syncthreads();   // the store has completed (thread 0 waited) before the next item's loads
}

// The persistent tensor-core kernel: one CTA per SM takes work items, the CTA
// tiles of the launch's jobs (items tile_begin[i] .. tile_begin[i+1] - 1 of
// job i, the jobs ordered by decreasing lattice side), from the launch's
// queue counter until none is left.  Lattices of every side share one launch,
// and a tile that takes longer (an MH recompute) delays only its own CTA's
// next pick instead of the end of a wave.  Tensor memory is allocated once
// per CTA; after an abort the CTA takes no further item.
template <int KT, int kT, bool EVAL>
__global__ void __launch_bounds__(kThr, 1) crbm_tc_kernel(const __grid_constant__ LaunchParams prm) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) unsigned long long s_bar[kNbar];
  __shared__ uint32_t s_tmem;
  __shared__ int s_item, s_abort;
  __shared__ uint8_t s_stage[32];
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) s_abort = 0;
  if (warp == 16) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" :: "r"(sm_addr(&s_tmem)),
                 "r"(kTmCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem, bar0 = sm_addr(s_bar);
  volatile int* abort = &s_abort;
  while (true) {
    if (tid == 0) s_item = *abort ? prm.total_items : atomicAdd(prm.queue, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= prm.total_items) break;
    int jid = 0;
    while (jid + 1 < prm.n_jobs && item >= prm.tile_begin[jid + 1]) ++jid;
    const JobDev& jb = prm.job[jid];
    const int t = item - prm.tile_begin[jid];
    if (jb.L == 128) tc_tile<128, KT, kT, EVAL>(prm, jb, t, smem, bar0, tmem, abort, s_stage);
    else if (jb.L == 64) tc_tile<64, KT, kT, EVAL>(prm, jb, 2 * t, smem, bar0, tmem, abort, s_stage);
    else if (jb.L == 32) tc_tile<32, KT, kT, EVAL>(prm, jb, 4 * t, smem, bar0, tmem, abort, s_stage);
    else tc_tile<16, KT, kT, EVAL>(prm, jb, 8 * t, smem, bar0, tmem, abort, s_stage);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 16)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" :: "r"(tmem), "r"(kTmCols));
}

// After a launch, in stream order (and in captured graphs): every job's step
// counter advances by S, and the queue counter is cleared for the next launch.
__global__ void tc_advance_kernel(const __grid_constant__ LaunchParams p) {
  const int i = threadIdx.x;
  if (i < p.n_jobs) *p.job[i].step += (unsigned long long)p.S;
  if (i == 0) *p.queue = 0;
}

// A bounded wait that runs out: one CTA waits for phase 0 of an mbarrier with
// the routine of the tensor-core pipeline (arrive = 1: after one arrival, so
// the wait succeeds at once; arrive = 0: nothing arrives, the wait gives up
// after `limit` cycles and raises the error flag).
__global__ void wait_probe_kernel(long long limit, int arrive, int* err) {
  __shared__ __align__(8) unsigned long long mb;
  __shared__ int ab;
  const uint32_t b = sm_addr(&mb);
  if (threadIdx.x == 0) {
    ab = 0;
    mbar_init(b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (arrive && threadIdx.x == 0) mbar_arrive(b);
  mbar_wait(b, 0u, limit, &ab, err);
}

template <int KT, int kT, bool EVAL>
cudaError_t tc_limit_inst(size_t bytes) {
  return cudaFuncSetAttribute(crbm_tc_kernel<KT, kT, EVAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int tc_chains_per_cta(int L) { return 128 / L; }

size_t tc_smem_bytes(int L, int K, int k) {
  return L == 128 ? tc_layout<128>(K, k).total
         : L == 64 ? tc_layout<64>(K, k).total
         : L == 32 ? tc_layout<32>(K, k).total
                   : tc_layout<16>(K, k).total;
}

bool tc_supported(int kind, int prec, int L, int K, int k) {
  return kind == kIsing && prec == kMixed && (L == 128 || L == 64 || L == 32 || L == 16) && K >= 1 && K <= 4 &&
         k >= 1 && k <= 5;
}

// One persistent launch for the jobs of p (one filter shape; any of the four
// sides), then the step counters and the queue counter.  p.mode 1: the
// evaluation of the current lattices (no proposal; step counters unchanged).
cudaError_t launch_tc(const LaunchParams& p, int grid, size_t smem, cudaStream_t st) {
  const bool eval = p.mode == 1;
  if ((!eval && p.S <= 0) || p.total_items <= 0) return cudaSuccess;
  const bool k45 = p.job[0].K == 4 && p.job[0].k == 5;
  if (eval) {
    if (k45) crbm_tc_kernel<4, 5, true><<<grid, kThr, smem, st>>>(p);
    else crbm_tc_kernel<0, 0, true><<<grid, kThr, smem, st>>>(p);
  } else {
    if (k45) crbm_tc_kernel<4, 5, false><<<grid, kThr, smem, st>>>(p);
    else crbm_tc_kernel<0, 0, false><<<grid, kThr, smem, st>>>(p);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    tc_advance_kernel<<<1, kMaxJobs, 0, st>>>(p);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t tc_set_smem_limit() {
  const size_t b = tc_layout<128>(4, 5).total;
  cudaError_t e = tc_limit_inst<4, 5, false>(b);
  if (e == cudaSuccess) e = tc_limit_inst<0, 0, false>(b);
  if (e == cudaSuccess) e = tc_limit_inst<4, 5, true>(b);
  if (e == cudaSuccess) e = tc_limit_inst<0, 0, true>(b);
  return e;
}

cudaError_t launch_wait_probe(long long limit, int arrive, int* err, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(limit, arrive, err);
  return cudaGetLastError();
}

}  // namespace crbm
