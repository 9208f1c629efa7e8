// libcholdiff host side: the C ABI of include/libcholdiff.h, the workspace
// arena, and the block-column schedulers that issue the blocked algorithms
// of Sec. 4.2 as grouped kernel launches on the caller's stream.
//
// Every operation is written once for a ragged batch of independent
// problems; a single call is a batch of one.  At each block step the work of
// all still-active problems goes into one grouped launch per kernel kind, so
// small problems share the GPU.
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <functional>
#include <vector>

#include "cd_internal.h"
#include "cd_mixed.h"

using namespace cd;

namespace {

constexpr int kDefaultNbSmall = 64;
constexpr int kDefaultNbLarge = 128;
constexpr size_t kPartBytes = size_t(64) << 20;  // split-K partial sums, per stream
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

struct Arena {
  char *base = nullptr;
  size_t cap = 0, off = 0;
  void *take(size_t bytes) {
    size_t o = align_up(off);
    if (o + bytes > cap) return nullptr;
    off = o + bytes;
    return base + o;
  }
};

// Default block sizes (measured on GB300, N = 8192).  The reverse and
// forward-sensitivity passes run fastest with 256-wide blocks at large n:
// split-BF16 ones are bound by their sequence of steps, and the FP64 ones
// gain a little (chol_rev 1.176 -> 1.185, chol_fwd_sens 1.152 -> 1.159
// TFLOP/s).  The factorisations (and the one-loop pass) prefer 128: their
// diagonal blocks (at most 128 wide) factorise on one cluster (FP64 chol_fwd 1.154 at
// 128, 1.088 at 256).
int pick_nb(int n, const cd_options *opt, bool factorisation = false) {
  int nb = (opt && opt->nb > 0) ? opt->nb : (n >= 1024 ? kDefaultNbLarge : kDefaultNbSmall);
  if (opt && opt->nb <= 0 && n >= 4096 && !factorisation) nb = 256;
  if (opt && opt->prec != CD_FP64) nb = (nb + 63) / 64 * 64;  // the tensor-core path works on 64-wide K blocks
  return nb;
}

int nblocks(int n, int nb) { return (n + nb - 1) / nb; }

// Workspace one problem of size n needs at one recursion level (dual: the
// one-loop factorisation-and-sensitivity pass, which keeps a second panel).
size_t prob_bytes(int n, int nb, bool dual = false) {
  if (n <= 0) return 0;
  return align_up(sizeof(double) * (size_t)nblocks(n, nb) * nb * nb) +
         (dual ? 2 : 1) * align_up(sizeof(double) * (size_t)n * nb) + 2 * align_up(sizeof(double) * (size_t)nb * nb);
}

// Extra workspace of the recursive diagonal step (nb > kTileMax).
size_t recursion_bytes(int nb) {
  if (nb <= kTileMax) return 0;
  return prob_bytes(nb, kTileMax, true) + align_up(sizeof(double) * (size_t)nb * nb) + 4 * kAlign;
}

struct Prob {
  int n;
  const double *L;  // factor (rev, sens); null for fwd
  long long ldl;
  double *X;  // in/out
  long long ldx;
  int *info;
  double *dinv;  // nblocks * nb * nb (ld nb)
  double *W;     // n * nb (ld nb)
  int col0;      // global column of this (sub)problem's first column (info)
  struct Mix {    // split-BF16 term arrays of the mixed path (null in FP64)
    void *big, *big2, *P1, *P2, *P3, *P4;
    void *P5;  // reverse pass: two block columns of C_bar side by side (n x 2 nb), for the deferred r2
    long long ldb, ldn;
    int pad, T;
    // CD_MIXED_FIXED4 factorisation: fixed-point slices of L (fbig, rows of L),
    // of the panel (fP1) and of D^{-1} (fP4, two slots used by step parity: the
    // diagonal tile writes step s's while the previous panel solve may still read
    // step s-1's), with their row exponents
    void *fbig, *fP1, *fP4;
    int *exL, *exP1, *exP4;
  } mx;
  double *T1, *T2;  // nb x nb temporaries of the symbolic diagonal step
  double *Xd;       // one-loop pass: tril(Sigma_dot) in, L_dot out (null otherwise)
  long long ldxd;
  double *W2;       // one-loop pass: the solved L_dot panel (n * nb, ld nb)
};

// Per-launch event records of cd_profile_enable.
struct Profiler {
  struct Rec {
    int kind;
    int side;  // launched on the handle's side stream
    cudaEvent_t e0, e1;
    double flops, bytes;
  };
  std::vector<std::string> names;
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  int kind_id(const char *name) {
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == name) return (int)i;
    names.emplace_back(name);
    return (int)names.size() - 1;
  }
  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  ~Profiler() {
    for (auto &r : recs) {
      cudaEventDestroy(r.e0);
      cudaEventDestroy(r.e1);
    }
    for (auto e : pool) cudaEventDestroy(e);
  }
};

struct Ctx {
  cd_handle *h;
  cudaStream_t s;
  const cd_options *opt;
  double *part;
  size_t part_cap;  // doubles
  int target_ctas;
  int err = CD_OK;
  cudaStream_t side = nullptr;  // second stream (null: everything on s)
  double *part2 = nullptr;      // split-K partials of work on the side stream
  size_t part2_cap = 0;
  double *part3 = nullptr, *part4 = nullptr;  // one-loop pass: the sensitivity steps' partials
  size_t part3_cap = 0;
  void check(cudaError_t e) {  // after a kernel launch
    ++h->launches;
    cuda(e);
  }
  void cuda(cudaError_t e) {  // after any other CUDA call
    if (e != cudaSuccess && err == CD_OK) {
      err = CD_ECUDA;
      if (getenv("CD_DEBUG")) fprintf(stderr, "libcholdiff: CUDA error %d (%s)\n", (int)e, cudaGetErrorString(e));
    }
  }
  // Launch through f(), recording an event pair around it when profiling.
  template <class F>
  void launch(const char *kind, double flops, double bytes, cudaStream_t st, F &&f) {
    Profiler *pr = h->prof_on ? (Profiler *)h->prof : nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (pr) {
      e0 = pr->ev();
      e1 = pr->ev();
      cudaEventRecord(e0, st);
    }
    const cudaError_t e = f();
    if (pr) {
      cudaEventRecord(e1, st);
      pr->recs.push_back({pr->kind_id(kind), (side && st == side) ? 1 : 0, e0, e1, flops, bytes});
    }
    check(e);
  }
  template <class F>
  void launch(const char *kind, double flops, double bytes, F &&f) {
    launch(kind, flops, bytes, s, f);
  }
  // Work enqueued on side() after fork() may run concurrently with work on s
  // until join() makes s wait for it.
  void fork() {
    if (!side) return;
    cuda(cudaEventRecord(h->ev_fork, s));
    cuda(cudaStreamWaitEvent(side, h->ev_fork, 0));
  }
  void join() {
    if (!side) return;
    cuda(cudaEventRecord(h->ev_join, side));
    cuda(cudaStreamWaitEvent(s, h->ev_join, 0));
  }
  // mark(): a point in the side stream's work so far; wait_mark(): s waits
  // for that point only (the side stream's later work may still run).
  void mark() {
    if (side) cuda(cudaEventRecord(h->ev_mid, side));
  }
  void wait_mark() {
    if (side) cuda(cudaStreamWaitEvent(s, h->ev_mid, 0));
  }
  // Named points in the side stream's work for the lookahead factorisation:
  // record one after the side-stream work that s will need, wait on it later.
  void record(cudaEvent_t e) {
    if (side) cuda(cudaEventRecord(e, side));
  }
  void wait(cudaEvent_t e) {
    if (side) cuda(cudaStreamWaitEvent(s, e, 0));
  }
};

// Products of at most this many multiply-adds use 32 x 32 output tiles.
constexpr double kSmallGemmWork = 67108864.0;

const char *kAName[6] = {"N", "T", "SYM2", "TL", "SYM1", "NL"};
const char *kBName[4] = {"N", "T", "TL", "NL"};

// Accumulates GEMMs of one kind into a grouped launch.  The split-K factor
// is chosen at flush time for the whole group so that the grid fills whole
// waves of resident CTAs (c.target_ctas), which keeps every SM's FP64 pipe
// busy to the end of the launch.
struct GemmBatch {
  Ctx &c;
  GemmGroup g;
  cudaStream_t st;
  double *part;
  size_t part_cap;
  GemmBatch(Ctx &ctx, int amode, int bmode, bool lower, bool on_side = false) : c(ctx) {
    memset(&g, 0, sizeof(g));
    g.amode = amode;
    g.bmode = bmode;
    g.lower = lower ? 1 : 0;
    const bool side = on_side && c.side;
    st = side ? c.side : c.s;
    part = side ? c.part2 : c.part;
    part_cap = side ? c.part2_cap : c.part_cap;
  }
  void add(int M, int N, int K, const double *A, long long lda, const double *B, long long ldb, const double *Cin,
           long long ldcin, double *Cout, long long ldcout, double alpha, double beta) {
    if (M <= 0 || N <= 0) return;
    if (K <= 0 && beta == 1.0 && Cin == Cout && ldcin == ldcout) return;  // identity update
    if (g.count == kMaxGemm) flush();
    GemmDesc &d = g.d[g.count++];
    d.A = A; d.B = B; d.Cin = Cin; d.Cout = Cout;
    d.lda = lda; d.ldb = ldb; d.ldcin = ldcin; d.ldcout = ldcout;
    d.alpha = alpha; d.beta = beta;
    d.M = M; d.N = N; d.K = K; d.splits = 1; d.kchunk = std::max(K, 1);
    d.tiles_m = (M + 63) / 64;
    d.tiles_n = (N + 63) / 64;
    d.part = nullptr;
  }
  int per_split(const GemmDesc &d) const { return g.lower ? d.tiles_m * (d.tiles_m + 1) / 2 : d.tiles_m * d.tiles_n; }
  // Output tile size of one problem, from its own shape: small products use
  // 32 x 32 tiles so that their work spreads over every SM's FP64 unit.
  int tile_size(const GemmDesc &d) const {
    const double outs = g.lower ? 0.5 * d.M * (d.M + 1.0) : (double)d.M * d.N;
    return outs * d.K <= kSmallGemmWork ? 32 : 64;
  }
  static double wave_eff(long long ctas, int slots) {
    const long long waves = (ctas + slots - 1) / slots;
    return (double)ctas / (double)(waves * slots);
  }
  // Split-K factor of one problem from its own shape only, so that a
  // problem gets the same arithmetic whether it runs alone or in a batch.
  int choose_splits(const GemmDesc &d, int ts) const {
    const int slots = std::max(1, ts == 32 ? c.h->gemm_slots_small : c.target_ctas);
    const long long t1 = per_split(d);
    if (t1 >= 4LL * slots || d.K < 32) return 1;
    const int smax = std::min(64, d.K / 16);
    int best = 1;
    double best_e = wave_eff(t1, slots);
    for (int s2 = 2; s2 <= smax && best_e < 0.9; ++s2) {
      const double e = wave_eff(t1 * s2, slots);
      if (e >= 0.9) return s2;
      if (e > best_e + 0.02) {
        best = s2;
        best_e = e;
      }
    }
    return best;
  }
  // The work items of a 32 x 32-tile group with triangular operands whose K
  // range is not empty (all items of problems without K splits, which write
  // their output even when it is zero); false if there are too many to list.
  static bool nonempty_items(const GemmGroup &sub, GemmItems &it) {
    it.count = 0;
    for (int p = 0; p < sub.count; ++p) {
      const GemmDesc &d = sub.d[p];
      const int per = sub.lower ? d.tiles_m * (d.tiles_m + 1) / 2 : d.tiles_m * d.tiles_n;
      for (int z = 0; z < d.splits; ++z)
        for (int rem = 0; rem < per; ++rem) {
          int ti, tj;
          if (sub.lower) {
            ti = 0;
            while ((ti + 1) * (ti + 2) / 2 <= rem) ++ti;
            tj = rem - ti * (ti + 1) / 2;
          } else {
            ti = rem / d.tiles_n;
            tj = rem % d.tiles_n;
          }
          const int m0 = ti * 32, n0 = tj * 32, kbeg = z * d.kchunk;
          int klo = kbeg, khi = std::min(d.K, kbeg + d.kchunk);
          if (sub.tri & TRI_A_UPPER) klo = std::max(klo, m0);
          if (sub.tri & TRI_B_LOWER) klo = std::max(klo, n0);
          if (sub.tri & TRI_A_LOWER) khi = std::min(khi, m0 + 32);
          if (sub.tri & TRI_B_UPPER) khi = std::min(khi, n0 + 32);
          if (d.splits > 1 && klo >= khi) continue;  // contributes nothing; its partial is not read
          if (it.count == kMaxItems) return false;
          it.bid[it.count++] = d.tile_begin + z * per + rem;
        }
    }
    return true;
  }
  void launch_sub(GemmGroup &sub, bool red, double flops, double bytes, double rbytes) {
    if (sub.count == 0) return;
    char name[48];
    snprintf(name, sizeof(name), "gemm_f64<%s,%s>%s%s%s", kAName[g.amode], kBName[g.bmode], g.lower ? "_tril" : "",
             g.phi ? "_phi" : "", sub.ts == 32 ? "_t32" : "");
    if (sub.ts == 32 && sub.tri && red) {
      static thread_local GemmItems it;
      if (nonempty_items(sub, it) && it.count < sub.total_tiles) {
        c.launch(name, flops, bytes, st, [&] { return launch_gemm_items(sub, it, st); });
        c.launch("splitk_reduce_f64", 0.0, rbytes, st, [&] { return launch_reduce_group(sub, st); });
        return;
      }
    }
    c.launch(name, flops, bytes, st, [&] { return launch_gemm_group(sub, st); });
    if (red) c.launch("splitk_reduce_f64", 0.0, rbytes, st, [&] { return launch_reduce_group(sub, st); });
  }
  // Whether to split the last r row (or column) tiles of a problem f times further along
  // K (a tail split): its CTAs carry equal work, one of them keeps its SM's
  // FP64 unit busy, and the launch lasts as long as the most loaded SM.  With
  // H whole units (tiles x splits) followed by T pieces of 1/f unit, handed
  // out in order to the least loaded SM, the span is computed in closed form
  // below; a tail split is taken when it is at least 3 % shorter.  The tail
  // is the last row tiles (A and C offset by rows) or, for A views that have
  // no row offset (the symmetric ones), the last column tiles (B and C offset
  // by columns).  Dense operands, general outputs and 64 x 64 tiles only; the
  // choice depends on the problem's shape alone.
  bool tail_split(const GemmDesc &d, int ts, int sp, int kchunk, int &r_out, int &f_out, bool &cols_out) const {
    if (ts != 64 || g.lower || g.tri) return false;
    const bool rows_ok = g.amode == A_N || g.amode == A_T;  // row tail: A and C offset by rows
    const bool cols_ok = g.bmode == B_N || g.bmode == B_T;  // column tail: B and C offset by columns
    if (!rows_ok && !cols_ok) return false;
    const long long S = std::max(1, c.h->num_sms);
    auto span = [&](long long H, long long T, int f) {
      const long long q = H / S, rem = H % S;
      if (T == 0) return (double)(rem ? q + 1 : q);
      if (rem == 0) return q + std::ceil((double)T / S) / f;
      const long long fill = (S - rem) * f;  // pieces that bring every SM to q + 1
      if (T <= fill) return (double)(q + 1);
      return q + 1 + std::ceil((double)(T - fill) / S) / f;
    };
    const long long units = (long long)d.tiles_m * d.tiles_n * sp;
    const double base = span(units, 0, 1);
    double best = base;
    int br = 0, bf = 1;
    bool bcols = false;
    for (int side = 0; side < 2; ++side) {
      const bool cols = side == 1;
      if (cols ? !cols_ok : !rows_ok) continue;
      const long long per = (long long)(cols ? d.tiles_m : d.tiles_n) * sp;  // units of one row (column) of tiles
      const int lines = cols ? d.tiles_n : d.tiles_m;
      for (int f = 2; f <= 8; ++f) {
        if (kchunk / f < 64) break;
        for (int r = 1; r <= lines; ++r) {
          const double v = span(units - r * per, r * per * f, f);
          if (v < best - 1e-9) {
            best = v;
            br = r;
            bf = f;
            bcols = cols;
          }
        }
      }
    }
    if (br == 0 || best > 0.97 * base) return false;
    r_out = br;
    f_out = bf;
    cols_out = bcols;
    return true;
  }
  // One launch (or more, if the partial region fills) per tile size.
  void flush_ts(int ts) {
    GemmGroup sub;
    memset(&sub, 0, sizeof(sub));
    sub.amode = g.amode;
    sub.bmode = g.bmode;
    sub.lower = g.lower;
    sub.phi = g.phi;
    sub.tri = g.tri;
    sub.ts = ts;
    const int ntri = ((g.tri & (TRI_A_UPPER | TRI_A_LOWER)) ? 1 : 0) + ((g.tri & (TRI_B_LOWER | TRI_B_UPPER)) ? 1 : 0);
    const double tri_frac = ntri == 0 ? 1.0 : (ntri == 1 ? 0.5 : 1.0 / 3.0);  // nonzero share of the K terms
    size_t used = 0;
    double flops = 0, bytes = 0, rbytes = 0;
    bool red = false;
    // one descriptor into the launch (partial region and descriptor slots permitting)
    auto emit = [&](GemmDesc d, int sp, int kchunk) {
      const size_t mn = (size_t)d.M * d.N;
      if ((sp > 1 && used + mn * sp > part_cap) || sub.count == kMaxGemm) {  // full: launch what we have first
        launch_sub(sub, red, flops, bytes, rbytes);
        sub.count = 0;
        sub.total_tiles = 0;
        used = 0;
        flops = bytes = rbytes = 0;
        red = false;
      }
      d.part = nullptr;
      if (sp > 1) {
        d.part = part + used;
        used += mn * sp;
      }
      d.splits = sp;
      d.kchunk = kchunk;
      d.tile_begin = sub.total_tiles;
      sub.total_tiles += per_split(d) * sp;
      sub.d[sub.count++] = d;
      const double outs = g.lower ? 0.5 * d.M * (d.M + 1.0) : (double)d.M * d.N;
      flops += 2.0 * d.K * outs * tri_frac;
      bytes += 8.0 * ((double)d.M * d.K + (double)d.K * d.N + outs * (d.beta != 0.0 ? 2.0 : 1.0));
      if (sp > 1) {
        red = true;
        rbytes += 8.0 * outs * (sp + (d.beta != 0.0 ? 2.0 : 1.0));
      }
    };
    for (int p = 0; p < g.count; ++p) {
      GemmDesc d = g.d[p];
      if (tile_size(d) != ts) continue;
      d.tiles_m = (d.M + ts - 1) / ts;
      d.tiles_n = (d.N + ts - 1) / ts;
      int sp = std::min(choose_splits(d, ts), std::max(1, d.K / 16));
      int kchunk = std::max(d.K, 1);
      if (sp > 1) {
        kchunk = ((d.K + sp - 1) / sp + 15) / 16 * 16;
        sp = (d.K + kchunk - 1) / kchunk;
      }
      const size_t mn = (size_t)d.M * d.N;
      if (sp > 1 && (!part || mn * sp > part_cap)) {  // as many splits as the partial region holds
        sp = part ? (int)std::max<size_t>(1, part_cap / mn) : 1;
        kchunk = sp > 1 ? ((d.K + sp - 1) / sp + 15) / 16 * 16 : std::max(d.K, 1);
        if (sp > 1) sp = (d.K + kchunk - 1) / kchunk;
      }
      // the last row tiles split further along K, so that every SM ends with
      // about the same work (see tail_split)
      int r = 0, f = 1;
      bool cols = false;
      if (tail_split(d, ts, sp, kchunk, r, f, cols) && part) {
        GemmDesc h = d, t = d;
        int head = 0;  // rows (columns) of the head; 0: the whole problem takes the finer split
        if (!cols) {
          head = (d.tiles_m - r) * ts;
          h.M = head;
          h.tiles_m = d.tiles_m - r;
          t.M = d.M - head;
          t.tiles_m = r;
          t.A = g.amode == A_N ? d.A + (long long)head * d.lda : d.A + head;
          if (d.Cin) t.Cin = d.Cin + (long long)head * d.ldcin;
          t.Cout = d.Cout + (long long)head * d.ldcout;
        } else {
          head = (d.tiles_n - r) * ts;
          h.N = head;
          h.tiles_n = d.tiles_n - r;
          t.N = d.N - head;
          t.tiles_n = r;
          t.B = g.bmode == B_N ? d.B + head : d.B + (long long)head * d.ldb;
          if (d.Cin) t.Cin = d.Cin + head;
          t.Cout = d.Cout + head;
        }
        const int kt = ((d.K + sp * f - 1) / (sp * f) + 15) / 16 * 16;
        const int st = (d.K + kt - 1) / kt;
        if ((size_t)t.M * t.N * st <= part_cap) {
          if (head > 0) emit(h, sp, kchunk);
          emit(t, st, kt);
          continue;
        }
      }
      emit(d, sp, kchunk);
    }
    launch_sub(sub, red, flops, bytes, rbytes);
  }
  void flush() {
    if (g.count == 0) return;
    flush_ts(64);
    flush_ts(32);
    g.count = 0;
    g.total_tiles = 0;
  }
  ~GemmBatch() { flush(); }
};

struct TileBatch {
  Ctx &c;
  TileOp op;
  TileGroup g;
  TileBatch(Ctx &ctx, TileOp o) : c(ctx), op(o) { memset(&g, 0, sizeof(g)); }
  void add(const TileDesc &d) {
    if (d.t <= 0) return;
    if (g.count == kMaxTile) flush();
    g.d[g.count++] = d;
  }
  void flush() {
    if (g.count == 0) return;
    static const char *names[5] = {"", "tile_rev", "tile_sens", "tile_trtri_cluster", "tile_potrf_cluster"};
    double flops = 0, bytes = 0;
    for (int p = 0; p < g.count; ++p) {
      const double t = g.d[p].t, tri = 0.5 * t * (t + 1) * 8.0;
      switch (op) {
        case T_REV: flops += 2.0 * t * t * t / 3.0; bytes += 3 * tri; break;
        case T_SENS: flops += 2.0 * t * t * t / 3.0; bytes += 3 * tri; break;
        case T_TRTRI: flops += t * t * t / 3.0; bytes += tri + 8 * t * t; break;
        case T_POTRF: flops += t * t * t / 3.0 * (g.d[p].inv ? 2.0 : 1.0); bytes += 2 * tri + (g.d[p].inv ? 8 * t * t : 0); break;
      }
    }
    g.err = c.h->dev_err;
    c.launch(names[op], flops, bytes, [&] { return launch_tile_group(op, g, c.s); });
    g.count = 0;
  }
  ~TileBatch() { flush(); }
};

// Accumulates the panel copies of all problems of one step into one launch.
struct CopyBatch {
  Ctx &c;
  CopyGroup g;
  double bytes = 0;
  bool subsym;  // dst -= tril(src + src^T) instead of dst = src
  explicit CopyBatch(Ctx &ctx, bool subsym_ = false) : c(ctx), subsym(subsym_) { memset(&g, 0, sizeof(g)); }
  void add(const double *src, long long lds, double *dst, long long ldd, int rows, int cols) {
    if (rows <= 0 || cols <= 0) return;
    if (g.count == kMaxCopy) flush();
    CopyDesc &d = g.d[g.count++];
    d.src = src; d.dst = dst; d.lds = lds; d.ldd = ldd; d.rows = rows; d.cols = cols;
    bytes += 16.0 * rows * cols;
  }
  void flush() {
    if (g.count == 0) return;
    if (subsym)
      c.launch("subsym_f64", 0.0, bytes, [&] { return launch_subsym_group(g, c.s); });
    else
      c.launch("copy_f64", 0.0, bytes, [&] { return launch_copy_group(g, c.s); });
    g.count = 0;
    bytes = 0;
  }
  ~CopyBatch() { flush(); }
};

TileDesc tdesc(const double *L, long long ldl, double *X, long long ldx, double *inv, long long ldinv, int t,
               int *info = nullptr, int col0 = 0) {
  TileDesc d;
  d.L = L; d.ldl = ldl; d.X = X; d.ldx = ldx; d.inv = inv; d.ldinv = ldinv;
  d.t = t; d.info = info; d.col0 = col0;
  d.fsl = nullptr; d.fex = nullptr; d.ldf = 0; d.frows = 0; d.fterms = 0;
  return d;
}

// The diagonal routine of the reverse and forward-sensitivity passes.  Both
// choices are exact (Sec. 4.2).  The products spread one block's work over
// many CTAs and measure faster on GB300 for multi-block problems; a problem
// that is a single tile (no panel work to overlap) is faster as one level-2
// CTA, batched with the others in one launch, and needs no block inverse.
// The choice depends on the problem alone, so a problem computes the same
// bits alone or batched.
bool diag_symbolic(const Ctx &c, const Prob &p, int nb) {
  const int d = c.opt ? c.opt->diag : CD_DIAG_AUTO;
  if (d == CD_DIAG_AUTO) return !(p.n <= nb && p.n <= kTileMax);
  return d != CD_DIAG_LEVEL2;
}

// One block of the reverse pass's diagonal step, Eq. symrevtril on the block:
// D_bar <- Phi(D^{-T} (P + P^T) D^{-1}),  P = Phi(D^T D_bar), with D^{-1} the
// precomputed inverse of the block (full storage, zeros above the diagonal).
struct DiagRev {
  const double *D;
  long long ldd;
  double *Db;
  long long lddb;
  const double *Dinv;
  double *T1, *T2;
  int w, ldt;
};
void rev_diag_symbolic(Ctx &c, const std::vector<DiagRev> &v) {
  {  // P = Phi(D^T D_bar)
    GemmBatch gb(c, A_TL, B_NL, true);
    gb.g.phi = 1;
    gb.g.tri = TRI_A_UPPER | TRI_B_LOWER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.D, x.ldd, x.Db, x.lddb, nullptr, 0, x.T1, x.ldt, 1.0, 0.0);
  }
  {  // Y = (P + P^T) D^{-1}   (D^{-1} lower)
    GemmBatch gb(c, A_SYM2, B_N, false);
    gb.g.tri = TRI_B_LOWER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.T1, x.ldt, x.Dinv, x.ldt, nullptr, 0, x.T2, x.ldt, 1.0, 0.0);
  }
  {  // D_bar = Phi(D^{-T} Y)   (D^{-T} upper)
    GemmBatch gb(c, A_T, B_N, true);
    gb.g.phi = 1;
    gb.g.tri = TRI_A_UPPER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.Dinv, x.ldt, x.T2, x.ldt, nullptr, 0, x.Db, x.lddb, 1.0, 0.0);
  }
}

// One block of the forward-sensitivity diagonal step, Eq. symfwd on the block:
// D_dot <- D Phi(D^{-1} S D^{-T}), S the symmetric block whose lower triangle
// is D_dot.
void sens_diag_symbolic(Ctx &c, const std::vector<DiagRev> &v) {
  {  // Z = S D^{-T}   (D^{-T} upper)
    GemmBatch gb(c, A_SYM1, B_T, false);
    gb.g.tri = TRI_B_UPPER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.Db, x.lddb, x.Dinv, x.ldt, nullptr, 0, x.T1, x.ldt, 1.0, 0.0);
  }
  {  // X = Phi(D^{-1} Z)   (D^{-1} lower)
    GemmBatch gb(c, A_N, B_N, true);
    gb.g.phi = 1;
    gb.g.tri = TRI_A_LOWER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.Dinv, x.ldt, x.T1, x.ldt, nullptr, 0, x.T2, x.ldt, 1.0, 0.0);
  }
  {  // D_dot = D X   (both lower)
    GemmBatch gb(c, A_NL, B_NL, true);
    gb.g.tri = TRI_A_LOWER | TRI_B_LOWER;
    for (auto &x : v) gb.add(x.w, x.w, x.w, x.D, x.ldd, x.T2, x.ldt, nullptr, 0, x.Db, x.lddb, 1.0, 0.0);
  }
}

// Forward declarations (recursive diagonal steps).
void run_fwd(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar, const std::function<void(int)> *after = nullptr,
             bool dinv_slots = false);
void run_rev(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar);
void run_sens(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar);
void run_dual(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar);

// inv (t x t, ld ldinv, zero above the diagonal) = tril(D)^{-1}.
// t <= kTileMax: one CTA; larger: split D = [D11 0; D21 D22] and use
// inv21 = -inv22 (D21 inv11).
void trtri_big(Ctx &c, const double *D, long long ldd, double *inv, long long ldinv, int t, Arena &ar) {
  if (t <= kTileMax) {
    TileBatch tb(c, T_TRTRI);
    tb.add(tdesc(D, ldd, nullptr, 0, inv, ldinv, t));
    return;
  }
  const int h1 = (t / 2 + 63) / 64 * 64, h2 = t - h1;
  trtri_big(c, D, ldd, inv, ldinv, h1, ar);
  trtri_big(c, D + (long long)h1 * ldd + h1, ldd, inv + (long long)h1 * ldinv + h1, ldinv, h2, ar);
  size_t mark = ar.off;
  double *T = (double *)ar.take(sizeof(double) * (size_t)h2 * h1);
  if (!T) { c.err = CD_ENOMEM; return; }
  {
    GemmBatch gb(c, A_N, B_N, false);  // T = D21 inv11
    gb.g.tri = TRI_B_LOWER;
    gb.add(h2, h1, h1, D + (long long)h1 * ldd, ldd, inv, ldinv, nullptr, 0, T, h1, 1.0, 0.0);
  }
  {
    GemmBatch gb(c, A_N, B_N, false);  // inv21 = -inv22 T  (inv22 lower, zero above)
    gb.g.tri = TRI_A_LOWER;
    gb.add(h2, h1, h2, inv + (long long)h1 * ldinv + h1, ldinv, T, h1, nullptr, 0, inv + (long long)h1 * ldinv,
           ldinv, -1.0, 0.0);
  }
  // inv12 = 0
  c.cuda(cudaMemset2DAsync(inv + h1, sizeof(double) * ldinv, 0, sizeof(double) * h2, h1, c.s));
  ar.off = mark;
}

// Diagonal block inverse for every block of a partition of each problem.
// rev_partition: blocks [max(0,k-nb), k) for k = n, n-nb, ... (short block
// first); otherwise [j, min(n, j+nb)) (short block last).
void precompute_dinv(Ctx &c, std::vector<Prob> &P, int nb, bool rev_partition, Arena &ar) {
  struct Blk {
    const double *D;
    long long ldd;
    double *inv;
    int w;
  };
  std::vector<Blk> two;  // kTileMax < w <= 2 kTileMax: one level of 2 x 2 blocking, batched
  {
    TileBatch tb(c, T_TRTRI);
    for (auto &p : P) {
      // the inverses serve the panel solves and the symbolic diagonal step only
      if (p.n <= nb && !diag_symbolic(c, p, nb)) continue;
      const int nbk = nblocks(p.n, nb);
      for (int s = 0; s < nbk; ++s) {
        int j, k;
        if (rev_partition) {
          k = p.n - s * nb;
          j = std::max(0, k - nb);
        } else {
          j = s * nb;
          k = std::min(p.n, j + nb);
        }
        const int w = k - j;
        double *inv = p.dinv + (size_t)s * nb * nb;
        const double *D = p.L + (long long)j * p.ldl + j;
        if (w <= kTileMax) {
          tb.add(tdesc(D, p.ldl, nullptr, 0, inv, nb, w));
        } else if (w <= 2 * kTileMax && 2 * ((w / 2 + 63) / 64 * 64) <= nb) {
          const int h1 = (w / 2 + 63) / 64 * 64;
          tb.add(tdesc(D, p.ldl, nullptr, 0, inv, nb, h1));
          tb.add(tdesc(D + (long long)h1 * p.ldl + h1, p.ldl, nullptr, 0, inv + (long long)h1 * nb + h1, nb, w - h1));
          two.push_back({D, p.ldl, inv, w});
        } else {
          tb.flush();
          trtri_big(c, D, p.ldl, inv, nb, w, ar);
        }
      }
    }
  }
  if (two.empty()) return;
  // [D11 0; D21 D22]^{-1} = [inv11 0; -inv22 D21 inv11  inv22]; the scratch
  // T = D21 inv11 (h2 x h1, h2 <= h1, 2 h1 <= nb) of every block goes to the
  // top-right quarter of its own nb x nb inverse buffer, cleared afterwards.
  {
    GemmBatch gb(c, A_N, B_N, false);
    gb.g.tri = TRI_B_LOWER;
    for (auto &b : two) {
      const int h1 = (b.w / 2 + 63) / 64 * 64, h2 = b.w - h1;
      gb.add(h2, h1, h1, b.D + (long long)h1 * b.ldd, b.ldd, b.inv, nb, nullptr, 0, b.inv + h1, nb, 1.0, 0.0);
    }
  }
  {
    GemmBatch gb(c, A_N, B_N, false);
    gb.g.tri = TRI_A_LOWER;
    for (auto &b : two) {
      const int h1 = (b.w / 2 + 63) / 64 * 64, h2 = b.w - h1;
      gb.add(h2, h1, h2, b.inv + (long long)h1 * nb + h1, nb, b.inv + h1, nb, nullptr, 0, b.inv + (long long)h1 * nb,
             nb, -1.0, 0.0);
    }
  }
  for (auto &b : two) {  // clear the top-right quarter (and the scratch beyond it) to zero
    const int h1 = (b.w / 2 + 63) / 64 * 64;
    c.cuda(cudaMemset2DAsync(b.inv + h1, sizeof(double) * nb, 0, sizeof(double) * (nb - h1), h1, c.s));
  }
}

bool bind_workspace(std::vector<Prob> &P, int nb, Arena &ar) {
  for (auto &p : P) {
    p.dinv = nullptr;
    p.W = p.W2 = nullptr;
    p.T1 = p.T2 = nullptr;
    if (p.n <= 0) continue;
    p.dinv = (double *)ar.take(sizeof(double) * (size_t)nblocks(p.n, nb) * nb * nb);
    p.W = (double *)ar.take(sizeof(double) * (size_t)p.n * nb);
    p.T1 = (double *)ar.take(sizeof(double) * (size_t)nb * nb);
    p.T2 = (double *)ar.take(sizeof(double) * (size_t)nb * nb);
    if (!p.dinv || !p.W || !p.T1 || !p.T2) return false;
    if (p.Xd) {
      p.W2 = (double *)ar.take(sizeof(double) * (size_t)p.n * nb);
      if (!p.W2) return false;
    }
  }
  return true;
}

// ------------------------------- chol_blocked (Sec. 4.2) -------------------
// after(s) and dinv_slots as in run_fwd_mixed (block column s of L is final on the chain).
void run_fwd(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar, const std::function<void(int)> *after,
             bool dinv_slots) {
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  for (int s = 0; s < steps && c.err == CD_OK; ++s) {
    c.fork();  // f3 does not depend on f1 / f2 of this step
    {  // f3: C <- C - B R^T
      GemmBatch gb(c, A_N, B_T, false, /*on_side=*/true);
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        double *C = p.X + (long long)k * p.ldx + j;
        gb.add(m, w, j, p.X + (long long)k * p.ldx, p.ldx, p.X + (long long)j * p.ldx, p.ldx, C, p.ldx, C, p.ldx,
               -1.0, 1.0);
      }
    }
    {  // f1: D <- D - tril(R R^T)
      GemmBatch gb(c, A_N, B_T, true);
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j;
        double *R = p.X + (long long)j * p.ldx;
        gb.add(w, w, j, R, p.ldx, R, p.ldx, R + j, p.ldx, R + j, p.ldx, -1.0, 1.0);
      }
    }
    const size_t slot = dinv_slots ? (size_t)s * nb * nb : 0;  // this block's D^{-1}
    {  // f2: D <- chol_unblocked(D); then the inverse of D for f4
      TileBatch tb(c, T_POTRF);  // factorisation and inverse of the diagonal block in one cluster launch
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j;
        double *D = p.X + (long long)j * p.ldx + j;
        if (w <= kTileMax) {
          tb.add(tdesc(nullptr, 0, D, p.ldx, (k < p.n || dinv_slots) ? p.dinv + slot : nullptr, nb, w, p.info,
                       p.col0 + j));
        } else {
          tb.flush();
          size_t mark = ar.off;
          std::vector<Prob> sub(1);
          sub[0] = Prob{w, nullptr, 0, D, p.ldx, p.info, nullptr, nullptr, p.col0 + j};
          if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
          run_fwd(c, sub, kTileMax, ar);
          trtri_big(c, D, p.ldx, p.dinv + slot, nb, w, ar);
          ar.off = mark;
        }
      }
      tb.flush();
    }
    c.join();
    {  // f4: C <- C tril(D)^{-T}   (W = C Dinv^T, then copy back)
      GemmBatch gb(c, A_N, B_T, false);
      gb.g.tri = TRI_B_UPPER;
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        gb.add(m, w, w, p.X + (long long)k * p.ldx + j, p.ldx, p.dinv + slot, nb, nullptr, 0, p.W, nb, 1.0, 0.0);
      }
    }
    {
      CopyBatch cb(c);
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        cb.add(p.W, nb, p.X + (long long)k * p.ldx + j, p.ldx, m, w);
      }
    }
    if (after) (*after)(s);
  }
}

// ------------------------------ chol_blocked_rev (Sec. 4.2) ----------------
void run_rev(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  precompute_dinv(c, P, nb, true, ar);
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  auto blk = [&](const Prob &p, int s, int &j, int &k) {
    k = p.n - s * nb;
    j = std::max(0, k - nb);
    return k > 0;
  };
  for (int s = 0; s < steps && c.err == CD_OK; ++s) {
    {  // r1: C_bar <- C_bar D^{-1}   (into W)
      GemmBatch gb(c, A_N, B_N, false);
      gb.g.tri = TRI_B_LOWER;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        gb.add(m, w, w, p.X + (long long)k * p.ldx + j, p.ldx, p.dinv + (size_t)s * nb * nb, nb, nullptr, 0, p.W,
               nb, 1.0, 0.0);
      }
    }
    {
      CopyBatch cb(c);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        cb.add(p.W, nb, p.X + (long long)k * p.ldx + j, p.ldx, m, w);
      }
    }
    c.fork();  // r2 writes B_bar only; r3, r4, r5 neither read nor write it
    {  // r2: B_bar <- B_bar - C_bar R
      GemmBatch gb(c, A_N, B_N, false, /*on_side=*/true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Bb = p.X + (long long)k * p.ldx;
        gb.add(m, j, w, p.W, nb, p.L + (long long)j * p.ldl, p.ldl, Bb, p.ldx, Bb, p.ldx, -1.0, 1.0);
      }
    }
    {  // r3: D_bar <- tril(D_bar) - tril(C_bar^T C)
      GemmBatch gb(c, A_T, B_N, true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Db = p.X + (long long)j * p.ldx + j;
        gb.add(w, w, m, p.W, nb, p.L + (long long)k * p.ldl + j, p.ldl, Db, p.ldx, Db, p.ldx, -1.0, 1.0);
      }
    }
    {  // r4 as the products of Eq. symrevtril (problems that use them)
      std::vector<DiagRev> v;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || !diag_symbolic(c, p, nb)) continue;
        v.push_back({p.L + (long long)j * p.ldl + j, p.ldl, p.X + (long long)j * p.ldx + j, p.ldx,
                     p.dinv + (size_t)s * nb * nb, p.T1, p.T2, k - j, nb});
      }
      if (!v.empty()) rev_diag_symbolic(c, v);
    }
    {  // r4: D_bar <- chol_unblocked_rev(D, D_bar)
      TileBatch tb(c, T_REV);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || diag_symbolic(c, p, nb)) continue;
        const int w = k - j;
        const double *D = p.L + (long long)j * p.ldl + j;
        double *Db = p.X + (long long)j * p.ldx + j;
        if (w <= kTileMax) {
          tb.add(tdesc(D, p.ldl, Db, p.ldx, nullptr, 0, w));
        } else {
          tb.flush();
          size_t mark = ar.off;
          std::vector<Prob> sub(1);
          sub[0] = Prob{w, D, p.ldl, Db, p.ldx, nullptr, nullptr, nullptr, 0};
          if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
          run_rev(c, sub, kTileMax, ar);
          ar.off = mark;
        }
      }
    }
    {  // r5: R_bar <- R_bar - C_bar^T B - (D_bar + D_bar^T) R  ==  R_bar - G L[j:n, 0:j]
      GemmBatch gb(c, A_SYM2, B_N, false);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j;
        double *Rb = p.X + (long long)j * p.ldx;
        gb.add(w, j, p.n - j, p.X + (long long)j * p.ldx + j, p.ldx, p.L + (long long)j * p.ldl, p.ldl, Rb, p.ldx,
               Rb, p.ldx, -1.0, 1.0);
      }
    }
    c.join();  // the next step's panel was written by r2 and r5
  }
}

// ------------------------------ chol_blocked_fwd (Sec. 4.2) ----------------
// One block step of chol_blocked_fwd (Sec. 4.2) in FP64: p.L the factor (block columns [0, j + nb)
// final), p.X the sensitivity L_dot, p.dinv's slot s the block's D^{-1}, p.W the panel scratch.
void sens_step(Ctx &c, std::vector<Prob> &P, int nb, int s, Arena &ar) {
  c.fork();  // g3 does not depend on g1 / g2 of this step
  for (int term = 0; term < 2; ++term) {  // g3: C_dot <- C_dot - B_dot R^T - B R_dot^T
    GemmBatch gb(c, A_N, B_T, false, /*on_side=*/true);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      double *Cd = p.X + (long long)k * p.ldx + j;
      if (term == 0)
        gb.add(m, w, j, p.X + (long long)k * p.ldx, p.ldx, p.L + (long long)j * p.ldl, p.ldl, Cd, p.ldx, Cd,
               p.ldx, -1.0, 1.0);
      else
        gb.add(m, w, j, p.L + (long long)k * p.ldl, p.ldl, p.X + (long long)j * p.ldx, p.ldx, Cd, p.ldx, Cd,
               p.ldx, -1.0, 1.0);
    }
  }
  for (int term = 0; term < 2; ++term) {  // g1: D_dot <- D_dot - tril(R_dot R^T + R R_dot^T)
    GemmBatch gb(c, A_N, B_T, true);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int w = std::min(p.n, j + nb) - j;
      const double *Rd = p.X + (long long)j * p.ldx;
      const double *R = p.L + (long long)j * p.ldl;
      double *Dd = p.X + (long long)j * p.ldx + j;
      if (term == 0)
        gb.add(w, w, j, Rd, p.ldx, R, p.ldl, Dd, p.ldx, Dd, p.ldx, -1.0, 1.0);
      else
        gb.add(w, w, j, R, p.ldl, Rd, p.ldx, Dd, p.ldx, Dd, p.ldx, -1.0, 1.0);
    }
  }
  {  // g2 as the products of Eq. symfwd (problems that use them)
    std::vector<DiagRev> v;
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n || !diag_symbolic(c, p, nb)) continue;
      const int w = std::min(p.n, j + nb) - j;
      v.push_back({p.L + (long long)j * p.ldl + j, p.ldl, p.X + (long long)j * p.ldx + j, p.ldx,
                   p.dinv + (size_t)s * nb * nb, p.T1, p.T2, w, nb});
    }
    if (!v.empty()) sens_diag_symbolic(c, v);
  }
  {  // g2: D_dot <- chol_unblocked_fwd(D, D_dot)
    TileBatch tb(c, T_SENS);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n || diag_symbolic(c, p, nb)) continue;
      const int w = std::min(p.n, j + nb) - j;
      const double *D = p.L + (long long)j * p.ldl + j;
      double *Dd = p.X + (long long)j * p.ldx + j;
      if (w <= kTileMax) {
        tb.add(tdesc(D, p.ldl, Dd, p.ldx, nullptr, 0, w));
      } else {
        tb.flush();
        size_t mark = ar.off;
        std::vector<Prob> sub(1);
        sub[0] = Prob{w, D, p.ldl, Dd, p.ldx, nullptr, nullptr, nullptr, 0};
        if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
        run_sens(c, sub, kTileMax, ar);
        ar.off = mark;
      }
    }
  }
  c.join();
  {  // g4a: C_dot <- C_dot - C D_dot^T
    GemmBatch gb(c, A_N, B_TL, false);
    gb.g.tri = TRI_B_UPPER;
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      double *Cd = p.X + (long long)k * p.ldx + j;
      gb.add(m, w, w, p.L + (long long)k * p.ldl + j, p.ldl, p.X + (long long)j * p.ldx + j, p.ldx, Cd, p.ldx, Cd,
             p.ldx, -1.0, 1.0);
    }
  }
  {  // g4b: C_dot <- C_dot D^{-T}   (into W, then copy back)
    GemmBatch gb(c, A_N, B_T, false);
    gb.g.tri = TRI_B_UPPER;
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      gb.add(m, w, w, p.X + (long long)k * p.ldx + j, p.ldx, p.dinv + (size_t)s * nb * nb, nb, nullptr, 0, p.W,
             nb, 1.0, 0.0);
    }
  }
  {
    CopyBatch cb(c);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      cb.add(p.W, nb, p.X + (long long)k * p.ldx + j, p.ldx, m, w);
    }
  }
}

void run_sens(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  precompute_dinv(c, P, nb, false, ar);
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  for (int s = 0; s < steps && c.err == CD_OK; ++s) sens_step(c, P, nb, s, ar);
}

// ------------- chol_blocked with chol_blocked_fwd in the same loop ----------
// Sec. 4.2 notes that the forward-mode updates can be accumulated while the
// factorisation is computed.  Step s finishes block column [j, k) of L (in X)
// and of L_dot (in Xd).  The bulk products f3 and g3 read only finished
// columns and run on the side stream; the chain f1, g1, f2, g2 runs on the
// high-priority stream; f4 and g4 then solve both panels with the one
// inverse of the new diagonal block.  A diagonal block wider than one tile
// is itself processed by this routine with tile-sized blocks.  (Used for
// blocks wider than one tile; run_dual pipelines the two passes otherwise.)
void run_dual_loop(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  auto blk = [&](const Prob &p, int s, int &j, int &k) {
    j = s * nb;
    k = std::min(p.n, j + nb);
    return j < p.n;
  };
  for (int s = 0; s < steps && c.err == CD_OK; ++s) {
    c.fork();
    {  // f1: D <- D - tril(R R^T);  g1, first term: D_dot <- D_dot - tril(R_dot R^T).
       // f1 and g1 are enqueued before the side stream's f3 and g3, so that their CTAs take SMs first.
      GemmBatch gb(c, A_N, B_T, true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j;
        const double *R = p.X + (long long)j * p.ldx, *Rd = p.Xd + (long long)j * p.ldxd;
        double *D = p.X + (long long)j * p.ldx + j, *Dd = p.Xd + (long long)j * p.ldxd + j;
        gb.add(w, w, j, R, p.ldx, R, p.ldx, D, p.ldx, D, p.ldx, -1.0, 1.0);
        gb.add(w, w, j, Rd, p.ldxd, R, p.ldx, Dd, p.ldxd, Dd, p.ldxd, -1.0, 1.0);
      }
    }
    {  // g1, second term: D_dot <- D_dot - tril(R R_dot^T)
      GemmBatch gb(c, A_N, B_T, true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j;
        double *Dd = p.Xd + (long long)j * p.ldxd + j;
        gb.add(w, w, j, p.X + (long long)j * p.ldx, p.ldx, p.Xd + (long long)j * p.ldxd, p.ldxd, Dd, p.ldxd, Dd,
               p.ldxd, -1.0, 1.0);
      }
    }
    {  // f3: C <- C - B R^T;  g3, first term: C_dot <- C_dot - B_dot R^T   (side stream)
      GemmBatch gb(c, A_N, B_T, false, /*on_side=*/true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *C = p.X + (long long)k * p.ldx + j, *Cd = p.Xd + (long long)k * p.ldxd + j;
        const double *R = p.X + (long long)j * p.ldx;
        gb.add(m, w, j, p.X + (long long)k * p.ldx, p.ldx, R, p.ldx, C, p.ldx, C, p.ldx, -1.0, 1.0);
        gb.add(m, w, j, p.Xd + (long long)k * p.ldxd, p.ldxd, R, p.ldx, Cd, p.ldxd, Cd, p.ldxd, -1.0, 1.0);
      }
    }
    {  // g3, second term: C_dot <- C_dot - B R_dot^T   (side stream)
      GemmBatch gb(c, A_N, B_T, false, /*on_side=*/true);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Cd = p.Xd + (long long)k * p.ldxd + j;
        gb.add(m, w, j, p.X + (long long)k * p.ldx, p.ldx, p.Xd + (long long)j * p.ldxd, p.ldxd, Cd, p.ldxd, Cd,
               p.ldxd, -1.0, 1.0);
      }
    }
    {  // f2: D <- chol_unblocked(D) and its inverse (wide blocks: both diagonal steps by recursion)
      TileBatch tb(c, T_POTRF);  // factorisation and inverse of the diagonal block in one cluster launch
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j;
        double *D = p.X + (long long)j * p.ldx + j;
        if (w <= kTileMax) {
          tb.add(tdesc(nullptr, 0, D, p.ldx, (k < p.n || diag_symbolic(c, p, nb)) ? p.dinv : nullptr, nb, w, p.info,
                       p.col0 + j));
        } else {
          tb.flush();
          size_t mark = ar.off;
          std::vector<Prob> sub(1);
          sub[0] = Prob{w, nullptr, 0, D, p.ldx, p.info, nullptr, nullptr, p.col0 + j};
          sub[0].Xd = p.Xd + (long long)j * p.ldxd + j;
          sub[0].ldxd = p.ldxd;
          if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
          run_dual_loop(c, sub, kTileMax, ar);
          if (k < p.n) trtri_big(c, D, p.ldx, p.dinv, nb, w, ar);
          ar.off = mark;
        }
      }
      tb.flush();
    }
    {  // g2 as the products of Eq. symfwd (problems that use them)
      std::vector<DiagRev> v;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || k - j > kTileMax || !diag_symbolic(c, p, nb)) continue;
        v.push_back({p.X + (long long)j * p.ldx + j, p.ldx, p.Xd + (long long)j * p.ldxd + j, p.ldxd, p.dinv, p.T1,
                     p.T2, k - j, nb});
      }
      if (!v.empty()) sens_diag_symbolic(c, v);
    }
    {  // g2: D_dot <- chol_unblocked_fwd(D, D_dot)
      TileBatch tb(c, T_SENS);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || k - j > kTileMax || diag_symbolic(c, p, nb)) continue;
        tb.add(tdesc(p.X + (long long)j * p.ldx + j, p.ldx, p.Xd + (long long)j * p.ldxd + j, p.ldxd, nullptr, 0,
                     k - j));
      }
    }
    c.join();
    {  // f4: W = C D^{-T}, the finished panel of L
      GemmBatch gb(c, A_N, B_T, false);
      gb.g.tri = TRI_B_UPPER;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        gb.add(m, w, w, p.X + (long long)k * p.ldx + j, p.ldx, p.dinv, nb, nullptr, 0, p.W, nb, 1.0, 0.0);
      }
    }
    {  // g4: W2 = (C_dot - W D_dot^T) D^{-T}, the finished panel of L_dot
      GemmBatch ga(c, A_N, B_TL, false);
      ga.g.tri = TRI_B_UPPER;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Cd = p.Xd + (long long)k * p.ldxd + j;
        ga.add(m, w, w, p.W, nb, p.Xd + (long long)j * p.ldxd + j, p.ldxd, Cd, p.ldxd, Cd, p.ldxd, -1.0, 1.0);
      }
      ga.flush();
      GemmBatch gb(c, A_N, B_T, false);
      gb.g.tri = TRI_B_UPPER;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        gb.add(m, w, w, p.Xd + (long long)k * p.ldxd + j, p.ldxd, p.dinv, nb, nullptr, 0, p.W2, nb, 1.0, 0.0);
      }
    }
    {
      CopyBatch cb(c);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        cb.add(p.W, nb, p.X + (long long)k * p.ldx + j, p.ldx, m, w);
        cb.add(p.W2, nb, p.Xd + (long long)k * p.ldxd + j, p.ldxd, m, w);
      }
    }
  }
}

// chol_blocked and chol_blocked_fwd (Sec. 4.1 takes both in one loop) in FP64: the factorisation
// as in run_fwd, each sensitivity step one block column behind it on a second chain and bulk
// stream, started by an event once the block column of L is final, with every block's D^{-1}
// in its slot of p.dinv and the sensitivity panel in W2.
void run_dual(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  cd_handle *h = c.h;
  if (nb > kTileMax || !h->crit2 || !h->side2 || !c.part3) {
    run_dual_loop(c, P, nb, ar);
    return;
  }
  std::vector<Prob> S = P;  // the sensitivity pass's view: L = the factor being formed, X = L_dot
  for (auto &q : S) {
    q.L = q.X;
    q.ldl = q.ldx;
    q.X = q.Xd;
    q.ldx = q.ldxd;
    q.W = q.W2;
    q.Xd = nullptr;
  }
  Ctx sc = c;
  sc.s = h->crit2;
  sc.side = h->side2;
  sc.part = c.part3;
  sc.part_cap = c.part3_cap;
  sc.part2 = c.part4;
  sc.part2_cap = c.part3_cap;
  c.cuda(cudaEventRecord(h->ev_start2, c.s));
  c.cuda(cudaStreamWaitEvent(sc.s, h->ev_start2, 0));
  const std::function<void(int)> after = [&](int s) {
    c.cuda(cudaEventRecord(h->ev_colA, c.s));
    c.cuda(cudaStreamWaitEvent(sc.s, h->ev_colA, 0));
    if (sc.err == CD_OK) sens_step(sc, S, nb, s, ar);
  };
  run_fwd(c, P, nb, ar, &after, true);
  sc.join();
  c.cuda(cudaEventRecord(h->ev_start2, sc.s));
  c.cuda(cudaStreamWaitEvent(c.s, h->ev_start2, 0));
  if (c.err == CD_OK && sc.err != CD_OK) c.err = sc.err;
}

// ============================================================================
// Mixed precision: the large off-diagonal products on the tensor cores with
// split-BF16 operands (cd_mixed.cu); diagonal tiles, their inverses and the
// Phi / halving steps stay in FP64 (the kernels above).
// ============================================================================
constexpr int kMixMaxChunk = 2048;  // longest FP32 accumulation before an FP64 reduction
constexpr int kMixMinKbPerSplit = 8;
constexpr int kFixedSlices = 4;  // CD_MIXED_FIXED4: fixed-point slices per operand
constexpr int kFixedMinKbPerSplit = 2;  // shortest K range (64-wide blocks) of one split-K part

MOp mop(void *base, long long ld, long long rows, int T, int x0, int y0) {
  MOp o;
  o.base = base;
  o.ld = ld;
  o.rows = rows;
  o.T = T;
  o.x0 = x0;
  o.y0 = y0;
  o.ex = nullptr;
  return o;
}

// A view of a fixed-point slice array (4 slices) with its row exponents.
MOp fop(void *base, long long ld, long long rows, const int *ex, int x0, int y0) {
  MOp o = mop(base, ld, rows, 4, x0, y0);
  o.ex = ex;
  return o;
}

void split(Ctx &c, cudaStream_t st, const double *src, long long lds, int rows, int cols, int mode, int transpose,
           void *dst, long long ldd, long long dst_rows, int reg_r0, int reg_c0, int h, int w, int dst_r0, int dst_c0,
           int T) {
  if (h <= 0 || w <= 0) return;
  SplitArgs a;
  a.src = src; a.lds = lds; a.rows = rows; a.cols = cols; a.mode = mode; a.transpose = transpose;
  a.dst = dst; a.ldd = ldd; a.dst_rows = dst_rows;
  a.reg_r0 = reg_r0; a.reg_c0 = reg_c0; a.dst_h = h; a.dst_w = w; a.dst_r0 = dst_r0; a.dst_c0 = dst_c0;
  a.T = T;
  a.ex = nullptr;
  c.launch("split_bf16", 0.0, (8.0 + 2.0 * T) * h * w, st, [&] { return mixed_split_group_launch(&a, 1, st, nullptr); });
}

// Accumulates the operand splits of all problems of one phase into grouped launches.
struct SplitBatch {
  Ctx &c;
  std::vector<SplitArgs> v;
  double bytes = 0;
  cudaStream_t st;
  explicit SplitBatch(Ctx &ctx, bool on_side = false) : c(ctx), st(on_side && ctx.side ? ctx.side : ctx.s) {}
  void add(const double *src, long long lds, int rows, int cols, int mode, int transpose, void *dst, long long ldd,
           long long dst_rows, int reg_r0, int reg_c0, int h, int w, int dst_r0, int dst_c0, int T) {
    if (h <= 0 || w <= 0) return;
    SplitArgs a;
    a.src = src; a.lds = lds; a.rows = rows; a.cols = cols; a.mode = mode; a.transpose = transpose;
    a.dst = dst; a.ldd = ldd; a.dst_rows = dst_rows;
    a.reg_r0 = reg_r0; a.reg_c0 = reg_c0; a.dst_h = h; a.dst_w = w; a.dst_r0 = dst_r0; a.dst_c0 = dst_c0;
    a.T = T;
    a.ex = nullptr;
    v.push_back(a);
    bytes += (8.0 + 2.0 * T) * h * w;
  }
  void flush() {
    if (v.empty()) return;
    c.launch("split_bf16", 0.0, bytes, st, [&] {
      int l = 0;
      const cudaError_t e = mixed_split_group_launch(v.data(), (int)v.size(), st, &l);
      if (l > 1) c.h->launches += l - 1;
      return e;
    });
    v.clear();
    bytes = 0;
  }
  ~SplitBatch() { flush(); }
};

// Fixed-point splits (4 slices) of all problems of one phase: with
// exponents computed from each destination row's region, or given.
struct FSplitBatch {
  Ctx &c;
  bool compute;
  std::vector<SplitArgs> v;
  double bytes = 0;
  cudaStream_t st;
  FSplitBatch(Ctx &ctx, bool compute_exponents, bool on_side = false)
      : c(ctx), compute(compute_exponents), st(on_side && ctx.side ? ctx.side : ctx.s) {}
  void add(const double *src, long long lds, int rows, int cols, int mode, void *dst, long long ldd,
           long long dst_rows, int reg_r0, int reg_c0, int h, int w, int dst_r0, int dst_c0, int *ex) {
    if (h <= 0 || w <= 0) return;
    SplitArgs a;
    a.src = src; a.lds = lds; a.rows = rows; a.cols = cols; a.mode = mode; a.transpose = 0;
    a.dst = dst; a.ldd = ldd; a.dst_rows = dst_rows;
    a.reg_r0 = reg_r0; a.reg_c0 = reg_c0; a.dst_h = h; a.dst_w = w; a.dst_r0 = dst_r0; a.dst_c0 = dst_c0;
    a.T = kFixedSlices;
    a.ex = ex;
    v.push_back(a);
    bytes += (8.0 * (compute ? 2 : 1) + 8.0) * h * w;
  }
  void flush() {
    if (v.empty()) return;
    c.launch("split_fixed4", 0.0, bytes, st, [&] {
      int l = 0;
      const cudaError_t e = fixed_split_group_launch(v.data(), (int)v.size(), compute, st, &l);
      if (l > 1) c.h->launches += l - 1;
      return e;
    });
    v.clear();
    bytes = 0;
  }
  ~FSplitBatch() { flush(); }
};

// Accumulates tensor-core products of one kind into grouped launches.
struct MixedBatch {
  Ctx &c;
  int T;
  bool lower;
  cudaStream_t st;
  double *part;
  size_t part_cap;
  static constexpr int kCap = 40;
  MProblem v[kCap];
  int count = 0;
  const char *tag;  // the algorithm step, for the profile
  bool fixed;       // fixed-point slice products (cd_fixed.cu); T is then 4
  MixedBatch(Ctx &ctx, int T_, bool lower_, bool on_side = false, const char *tag_ = nullptr, bool fixed_ = false)
      : c(ctx), T(T_), lower(lower_), tag(tag_), fixed(fixed_) {
    const bool side = on_side && c.side;
    st = side ? c.side : c.s;
    part = side ? c.part2 : c.part;
    part_cap = side ? c.part2_cap : c.part_cap;
  }
  void add(const MOp &A, const MOp &B, int M, int N, int K, const double *Cin, long long ldcin, double *Cout,
           long long ldcout, double alpha, double beta) {
    if (M <= 0 || N <= 0 || K <= 0) return;
    if (count == kCap) flush();
    MProblem &P = v[count++];
    P.A = A; P.B = B; P.M = M; P.N = N; P.K = K;
    P.Cin = Cin; P.ldcin = ldcin; P.Cout = Cout; P.ldcout = ldcout;
    P.alpha = alpha; P.beta = beta; P.part = nullptr; P.splits = 1; P.kchunk = (K + 63) / 64 * 64;
  }
  static double wave_eff(long long ctas, int slots) {
    const long long waves = (ctas + slots - 1) / slots;
    return (double)ctas / (double)(waves * slots);
  }
  int choose_splits(const MProblem &P) const {
    const int slots = std::max(1, c.h->num_sms * mixed_ctas_per_sm());
    const int tm = (P.M + 127) / 128, tn = fixed ? (P.N + 63) / 64 : (P.N + 127) / 128;
    long long t1 = lower ? tm * (tm + 1) / 2 : tm * tn;
    if (fixed && lower) {
      t1 = 0;
      for (int ti = 0; ti < tm; ++ti) t1 += std::min(tn, 2 * ti + 2);
    }
    const int kblocks = (P.K + 63) / 64;
    int sg = 1;
    if (t1 < 4LL * slots) {
      // each split keeps at least kMixMinKbPerSplit K blocks: a CTA's fixed
      // cost and the FP32 partial traffic outweigh finer parallelism
      // (fixed-point products: their 64-bit partials are exact and cheap to
      // sum, so a split may be as short as kFixedMinKbPerSplit blocks)
      const int smax = std::min(64, std::max(1, kblocks / (fixed ? kFixedMinKbPerSplit : kMixMinKbPerSplit)));
      double best = wave_eff(t1, slots);
      for (int s2 = 2; s2 <= smax && best < 0.9; ++s2) {
        const double e = wave_eff(t1 * s2, slots);
        if (e > best + 0.02) { sg = s2; best = e; }
      }
    }
    if (fixed) return std::min(sg, kblocks);  // exact over any K: splits only for parallelism
    return std::max((P.K + kMixMaxChunk - 1) / kMixMaxChunk, std::min(sg, kblocks));
  }
  void launch_range(int b, int e, double flops, double bytes) {
    if (e <= b) return;
    const int prods = fixed ? 13 : T == 3 ? 6 : 3;
    char name[48];
    snprintf(name, sizeof(name), "%s%d%s%s%s", fixed ? "fgemm_fixed4x" : "mgemm_bf16x", prods, lower ? "_tril" : "",
             tag ? " " : "", tag ? tag : "");
    c.launch(name, flops, bytes, st, [&] {
      int l = 0;
      const bool bulk = c.side && st == c.side;
      const int mu = bulk ? kUnitsPerCtaBulk : kUnitsPerCtaChain;
      cudaError_t err = fixed ? fixed_gemm_launch(v + b, e - b, lower, c.h->dev_err, st, &l, 2 * mu)
                              : mixed_gemm_launch(v + b, e - b, T, lower, c.h->dev_err, st, &l, 0, mu);
      if (l > 1) c.h->launches += l - 1;
      return err;
    });
  }
  void flush() {
    if (count == 0) return;
    size_t used = 0;
    double flops = 0, bytes = 0;
    const int prods = fixed ? 13 : T == 3 ? 6 : 3;
    int begin = 0;
    for (int i = 0; i < count; ++i) {
      MProblem &P = v[i];
      const int kblocks = (P.K + 63) / 64;
      int sp = choose_splits(P);
      int kchunk = ((kblocks + sp - 1) / sp) * 64;
      sp = (P.K + kchunk - 1) / kchunk;
      const size_t mn = (size_t)P.M * P.N;
      if (sp > 1 && (!part || mn * sp > part_cap)) {  // as many splits as the partial region holds
        sp = part ? (int)std::max<size_t>(1, part_cap / mn) : 1;
        kchunk = ((kblocks + sp - 1) / sp) * 64;
        sp = (P.K + kchunk - 1) / kchunk;
      }
      if (sp > 1 && used + mn * sp > part_cap) {
        launch_range(begin, i, flops, bytes);
        begin = i;
        used = 0;
        flops = bytes = 0;
      }
      P.part = nullptr;
      if (sp > 1) {
        P.part = part + used;
        used += mn * sp;
      }
      P.splits = sp;
      P.kchunk = kchunk;
      const double outs = lower ? 0.5 * P.M * (P.M + 1.0) : (double)P.M * P.N;
      flops += 2.0 * prods * P.K * outs;  // tensor-core flops (all term products)
      bytes += 2.0 * T * ((double)P.M * P.K + (double)P.N * P.K) + outs * 8.0 * (P.beta != 0.0 ? 2.0 : 1.0);
    }
    launch_range(begin, count, flops, bytes);
    count = 0;
  }
  ~MixedBatch() { flush(); }
};

// Split-BF16 terms of the products (CD_MIXED_FIXED4 keeps the three-term
// split for the derivative passes and fixed-point slices for the factor).
int mix_terms(int prec) { return prec == CD_MIXED_BF16X3 ? 2 : 3; }
size_t fixed_bytes(int n, int nb) {
  if (n <= 0) return 0;
  const size_t ldb = (size_t)((n + 63) / 64 * 64);
  const size_t e = (size_t)n * ldb + (size_t)n * nb + 2 * (size_t)nb * nb;  // fP4: two slots
  return 2 * (size_t)kFixedSlices * e + sizeof(int) * (2 * (size_t)n + 2 * nb) + 8 * kAlign;
}

size_t mix_bytes(int n, int nb, int T, bool two_big, bool fixed = false, bool rev = false) {
  if (n <= 0) return 0;
  const size_t ldb = (size_t)((n + 8 + 63) / 64 * 64), ldn = (size_t)((n + 63) / 64 * 64 + 64);
  const size_t e = (two_big ? 2 : 1) * (size_t)n * ldb + (size_t)n * nb + 2 * (size_t)nb * ldn + 2 * (size_t)nb * nb +
                   (rev ? 2 * (size_t)n * nb : 0);
  return 2 * (size_t)T * e + 9 * kAlign + (fixed ? fixed_bytes(n, nb) : 0);
}

bool bind_mixed(std::vector<Prob> &P, int nb, int T, bool two_big, Arena &ar, bool fixed = false, bool rev = false) {
  for (auto &p : P) {
    memset(&p.mx, 0, sizeof(p.mx));
    if (p.n <= 0) continue;
    const long long n = p.n;
    p.mx.T = T;
    p.mx.ldb = (n + 8 + 63) / 64 * 64;
    p.mx.ldn = (n + 63) / 64 * 64 + 64;
    p.mx.pad = (int)((8 - n % 8) % 8);
    const size_t t = 2 * (size_t)T;
    p.mx.big = ar.take(t * n * p.mx.ldb);
    p.mx.big2 = two_big ? ar.take(t * n * p.mx.ldb) : nullptr;
    p.mx.P1 = ar.take(t * n * nb);
    p.mx.P2 = ar.take(t * nb * p.mx.ldn);
    p.mx.P3 = ar.take(t * nb * p.mx.ldn);
    p.mx.P4 = ar.take(2 * t * nb * nb);  // two slots: the factorisation's D^{-1} by step parity
    p.mx.P5 = rev ? ar.take(t * n * 2 * nb) : nullptr;
    if (!p.mx.big || (two_big && !p.mx.big2) || !p.mx.P1 || !p.mx.P2 || !p.mx.P3 || !p.mx.P4 || (rev && !p.mx.P5))
      return false;
    if (fixed) {
      const size_t f = 2 * (size_t)kFixedSlices, ldf = (size_t)((n + 63) / 64 * 64);
      p.mx.fbig = ar.take(f * n * ldf);
      p.mx.fP1 = ar.take(f * n * nb);
      p.mx.fP4 = ar.take(2 * f * nb * nb);  // two slots, by step parity
      p.mx.exL = (int *)ar.take(sizeof(int) * n);
      p.mx.exP1 = (int *)ar.take(sizeof(int) * n);
      p.mx.exP4 = (int *)ar.take(sizeof(int) * 2 * nb);
      if (!p.mx.fbig || !p.mx.fP1 || !p.mx.fP4 || !p.mx.exL || !p.mx.exP1 || !p.mx.exP4) return false;
    }
  }
  return true;
}

// chol_blocked_rev (Sec. 4.2), products in split BF16.  L^T is split once
// (columns shifted by pad so that every block boundary is a multiple of 8).
//
// r2 (B_bar <- B_bar - C_bar R) is deferred every other step ("the partitioning is arbitrary",
// Sec. 4.2): an even step applies its C_bar R only to the block column of B_bar the next step
// reads as its C_bar, and the next (odd) step applies both steps' parts to the rest in one
// product with K = 2 nb, the two C_bar blocks side by side (columns [j, k + nb) of Sigma_bar,
// split into P5).  B_bar's FP64 read-modify-write then happens once every two steps.
void run_rev_mixed(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  precompute_dinv(c, P, nb, true, ar);
  {
    SplitBatch sb(c);
    for (auto &p : P) {
      const auto &x = p.mx;
      sb.add(p.L, p.ldl, p.n, p.n, 1, 1, x.big, x.ldb, p.n, 0, 0, p.n, (int)x.ldb, 0, x.pad, x.T);
    }
  }
  const int T = P.empty() ? 2 : P[0].mx.T;
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  auto blk = [&](const Prob &p, int s, int &j, int &k) {
    k = p.n - s * nb;
    j = std::max(0, k - nb);
    return k > 0;
  };
  for (int s = 0; s < steps && c.err == CD_OK; ++s) {
    const bool odd = s % 2 == 1;  // this step also applies the previous step's deferred r2
    {  // r1: C_bar <- C_bar D^{-1} (from the split copy of C_bar, so in place); then C_bar and C_bar^T split for r2, r3
      {
        SplitBatch sb(c);
        for (auto &p : P) {
          int j, k;
          if (!blk(p, s, j, k)) continue;
          const int w = k - j, m = p.n - k;
          if (m <= 0) continue;
          sb.add(p.X + (long long)k * p.ldx + j, p.ldx, m, w, 0, 0, p.mx.P1, nb, p.n, 0, 0, m, nb, 0, 0, T);
          sb.add(p.dinv + (size_t)s * nb * nb, nb, w, w, 0, 1, p.mx.P4, nb, nb, 0, 0, nb, nb, 0, 0, T);
        }
      }
      MixedBatch mb(c, T, false, false, "r1");
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Cb = p.X + (long long)k * p.ldx + j;
        mb.add(mop(p.mx.P1, nb, p.n, T, 0, 0), mop(p.mx.P4, nb, nb, T, 0, 0), m, w, w, nullptr, 0, Cb, p.ldx, 1.0,
               0.0);
      }
    }
    {
      SplitBatch sb(c);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        if (m <= 0) continue;
        const double *Cb = p.X + (long long)k * p.ldx + j;
        sb.add(Cb, p.ldx, m, w, 0, 0, p.mx.P1, nb, p.n, 0, 0, m, nb, 0, 0, T);
        // C_bar^T is the K = m operand of r3 and r5a: its columns up to the next
        // 64-wide K block are written (zeros past m), the rest is never read
        const int kw = (int)std::min<long long>(p.mx.ldn, (m + 63) / 64 * 64);
        sb.add(Cb, p.ldx, m, w, 0, 1, p.mx.P2, p.mx.ldn, nb, 0, 0, w, kw, 0, 0, T);
        // odd step: the rows below the previous block, this C_bar and the previous one side by side
        const int kp = std::min(p.n, k + nb);
        if (odd && j > 0 && kp < p.n && p.mx.P5)
          sb.add(p.X + (long long)kp * p.ldx + j, p.ldx, p.n - kp, kp - j, 0, 0, p.mx.P5, 2 * nb, p.n, 0, 0,
                 p.n - kp, 2 * nb, 0, 0, T);
      }
    }
    c.fork();
    {  // r3: D_bar <- tril(D_bar) - tril(C_bar^T C).  Enqueued before the side stream's
       // products so that its few CTAs take SMs first.
      MixedBatch mb(c, T, true, false, "r3");
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k)) continue;
        const int w = k - j, m = p.n - k;
        double *Db = p.X + (long long)j * p.ldx + j;
        mb.add(mop(p.mx.P2, p.mx.ldn, nb, T, 0, 0), mop(p.mx.big, p.mx.ldb, p.n, T, k + p.mx.pad, j), w, w, m, Db,
               p.ldx, Db, p.ldx, -1.0, 1.0);
      }
    }
    {  // r5, first part (side stream): R_bar <- R_bar - C_bar^T B.  It needs
       // neither r3 nor r4, so it leaves the diagonal chain.
      MixedBatch mb(c, T, false, true, "r5a");
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || j == 0) continue;
        const int w = k - j, m = p.n - k;
        double *Rb = p.X + (long long)j * p.ldx;
        mb.add(mop(p.mx.P2, p.mx.ldn, nb, T, 0, 0), mop(p.mx.big, p.mx.ldb, p.n, T, k + p.mx.pad, 0), w, j, m, Rb,
               p.ldx, Rb, p.ldx, -1.0, 1.0);
      }
    }
    c.mark();  // r5's second part waits for this point only
    {  // r2 (side stream): B_bar <- B_bar - C_bar R, deferred every other step (see above)
      MixedBatch mb(c, T, false, true, "r2");
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || j == 0) continue;
        const int w = k - j, m = p.n - k;
        const MOp C = mop(p.mx.P1, nb, p.n, T, 0, 0);
        if (!p.mx.P5) {  // no deferral
          mb.add(C, mop(p.mx.big, p.mx.ldb, p.n, T, j + p.mx.pad, 0), m, j, w, p.X + (long long)k * p.ldx, p.ldx,
                 p.X + (long long)k * p.ldx, p.ldx, -1.0, 1.0);
        } else if (!odd) {  // only columns [j - nb, j), which the next step reads; the rest waits
          const int j0 = std::max(0, j - nb);
          double *Bb = p.X + (long long)k * p.ldx + j0;
          mb.add(C, mop(p.mx.big, p.mx.ldb, p.n, T, j + p.mx.pad, j0), m, j - j0, w, Bb, p.ldx, Bb, p.ldx, -1.0,
                 1.0);
        } else {
          const int kp = std::min(p.n, k + nb);
          double *Bb = p.X + (long long)k * p.ldx;
          // rows [k, kp) (the previous block's rows): this step's part only
          mb.add(C, mop(p.mx.big, p.mx.ldb, p.n, T, j + p.mx.pad, 0), kp - k, j, w, Bb, p.ldx, Bb, p.ldx, -1.0, 1.0);
          // rows [kp, n): this step's part and the previous step's deferred one, K = kp - j
          if (kp < p.n) {
            double *Bb2 = p.X + (long long)kp * p.ldx;
            mb.add(mop(p.mx.P5, 2 * nb, p.n, T, 0, 0), mop(p.mx.big, p.mx.ldb, p.n, T, j + p.mx.pad, 0), p.n - kp, j,
                   kp - j, Bb2, p.ldx, Bb2, p.ldx, -1.0, 1.0);
          }
        }
      }
    }
    {  // r4 as the products of Eq. symrevtril (problems that use them)
      std::vector<DiagRev> v;
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || !diag_symbolic(c, p, nb)) continue;
        v.push_back({p.L + (long long)j * p.ldl + j, p.ldl, p.X + (long long)j * p.ldx + j, p.ldx,
                     p.dinv + (size_t)s * nb * nb, p.T1, p.T2, k - j, nb});
      }
      if (!v.empty()) rev_diag_symbolic(c, v);
    }
    {  // r4: D_bar <- chol_unblocked_rev(D, D_bar)   (FP64)
      TileBatch tb(c, T_REV);
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || diag_symbolic(c, p, nb)) continue;
        const int w = k - j;
        const double *D = p.L + (long long)j * p.ldl + j;
        double *Db = p.X + (long long)j * p.ldx + j;
        if (w <= kTileMax) {
          tb.add(tdesc(D, p.ldl, Db, p.ldx, nullptr, 0, w));
        } else {
          tb.flush();
          size_t mark = ar.off;
          std::vector<Prob> sub(1);
          sub[0] = Prob{w, D, p.ldl, Db, p.ldx, nullptr, nullptr, nullptr, 0};
          if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
          run_rev(c, sub, kTileMax, ar);
          ar.off = mark;
        }
      }
    }
    {  // r5, second part: R_bar <- R_bar - (D_bar + D_bar^T) R, after r4 and the first part
      {
        SplitBatch sb(c);
        for (auto &p : P) {
          int j, k;
          if (!blk(p, s, j, k) || j == 0) continue;
          const int w = k - j;
          sb.add(p.X + (long long)j * p.ldx + j, p.ldx, w, w, 2, 0, p.mx.P3, p.mx.ldn, nb, 0, 0, w,
                (w + 63) / 64 * 64, 0, 0, T);
        }
      }
      c.wait_mark();
      MixedBatch mb(c, T, false, false, "r5b");
      for (auto &p : P) {
        int j, k;
        if (!blk(p, s, j, k) || j == 0) continue;
        const int w = k - j;
        double *Rb = p.X + (long long)j * p.ldx;
        mb.add(mop(p.mx.P3, p.mx.ldn, nb, T, 0, 0), mop(p.mx.big, p.mx.ldb, p.n, T, j + p.mx.pad, 0), w, j, w, Rb,
               p.ldx, Rb, p.ldx, -1.0, 1.0);
      }
    }
    c.join();
  }
}

// chol_blocked (Sec. 4.2), products in split BF16; the finished columns of L
// are split into `big` block column by block column.
// after(s), if given, is called once block column s of L is final on both streams (the one-loop
// pass hangs its sensitivity step there); dinv_slots keeps every block's D^{-1} (slot s of
// p.dinv, the last block's too) instead of reusing slot 0.
void run_fwd_mixed(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar,
                   const std::function<void(int)> *after = nullptr, bool dinv_slots = false) {
  const int T = P.empty() ? 2 : P[0].mx.T;
  const bool fx = c.opt->prec == CD_MIXED_FIXED4;
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  if (fx)  // row exponents of L from the diagonal of Sigma, before it is overwritten
    for (auto &p : P)
      c.launch("diag_exponents", 0.0, 12.0 * p.n,
               [&] { return fixed_diag_exponents(p.X, p.ldx, p.n, p.mx.exL, c.s); });
  auto Lop = [&](const Prob &p, int x0, int y0) {
    return fx ? fop(p.mx.fbig, (p.n + 63) / 64 * 64, p.n, p.mx.exL, x0, y0) : mop(p.mx.big, p.mx.ldb, p.n, T, x0, y0);
  };
  // Lookahead.  Block column t is updated from the finished columns [0, j_t)
  // in two parts: from [0, j_t - nb) on the side stream one step early,
  // beside the diagonal tile of step t - 1 (f1 "old" and f3 "old"), and from
  // the previous block column [j_t - nb, j_t) once it is split (f1 "new" on
  // the chain, f3 "new" on the side stream).  The chain of a step is then
  // the rank-nb update of the diagonal block, its factorisation, the panel
  // solve and the split; the K = j_t products leave it.
  auto upd = [&](int t, int k0, int k1, bool on_side, bool want_f1, bool want_f3) {
    if (k1 <= k0) return;
    if (want_f1) {
      MixedBatch mb(c, T, true, on_side, "f1", fx);
      for (auto &p : P) {
        const int j = t * nb;
        if (j >= p.n) continue;
        const int w = std::min(p.n, j + nb) - j;
        double *D = p.X + (long long)j * p.ldx + j;
        mb.add(Lop(p, k0, j), Lop(p, k0, j), w, w, k1 - k0, D, p.ldx, D, p.ldx, -1.0, 1.0);
      }
    }
    if (want_f3) {
      MixedBatch mb(c, T, false, on_side, "f3", fx);
      for (auto &p : P) {
        const int j = t * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        double *C = p.X + (long long)k * p.ldx + j;
        mb.add(Lop(p, k0, k), Lop(p, k0, j), m, w, k1 - k0, C, p.ldx, C, p.ldx, -1.0, 1.0);
      }
    }
  };
  // f4's panel operand: the panel C of block column t (final once f3 is done), split for the
  // product with D^{-1}; it does not wait for the diagonal factorisation
  auto split_panel = [&](int t, bool on_side) {
    if (fx) {
      FSplitBatch sb(c, true, on_side);
      for (auto &p : P) {
        const int jj = t * nb;
        if (jj >= p.n) continue;
        const int k = std::min(p.n, jj + nb), w = k - jj, m = p.n - k;
        if (m <= 0) continue;
        sb.add(p.X + (long long)k * p.ldx + jj, p.ldx, m, w, 0, p.mx.fP1, nb, p.n, 0, 0, m, nb, 0, 0, p.mx.exP1);
      }
    } else {
      SplitBatch sb(c, on_side);
      for (auto &p : P) {
        const int jj = t * nb;
        if (jj >= p.n) continue;
        const int k = std::min(p.n, jj + nb), w = k - jj, m = p.n - k;
        if (m <= 0) continue;
        sb.add(p.X + (long long)k * p.ldx + jj, p.ldx, m, w, 0, 0, p.mx.P1, nb, p.n, 0, 0, m, nb, 0, 0, T);
      }
    }
  };
  // step t's D^{-1} slices and exponents (fixed4): slot t % 2
  auto fP4s = [&](const Prob &p, int t) {
    return (void *)((char *)p.mx.fP4 + (size_t)(t & 1) * 2 * kFixedSlices * nb * nb);
  };
  auto exP4s = [&](const Prob &p, int t) { return p.mx.exP4 + (size_t)(t & 1) * nb; };
  // the same for the three-term split: the previous panel solve may still read step t-1's
  auto P4s = [&](const Prob &p, int t) { return (void *)((char *)p.mx.P4 + (size_t)(t & 1) * 2 * T * nb * nb); };
  bool look_set[2] = {false, false};
  for (int s = 0; s < steps && c.err == CD_OK; ++s) {
    const int j = s * nb;
    const size_t slot = dinv_slots ? (size_t)s * nb * nb : 0;  // this block's D^{-1}
    {  // f2: D <- chol_unblocked(D), then D^{-1}   (FP64)
      TileBatch tb(c, T_POTRF);  // factorisation and inverse of the diagonal block in one cluster launch
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int w = std::min(p.n, j + nb) - j;
        double *D = p.X + (long long)j * p.ldx + j;
        if (w <= kTileMax) {
          TileDesc td = tdesc(nullptr, 0, D, p.ldx, (j + w < p.n || dinv_slots) ? p.dinv + slot : nullptr, nb, w,
                              p.info, p.col0 + j);
          if (j + w < p.n && nb <= kTileMax) {  // D^{-1} straight into the panel solve's operand
            td.fsl = fx ? fP4s(p, s) : P4s(p, s);
            td.fex = fx ? exP4s(p, s) : nullptr;
            td.fterms = fx ? 0 : T;
            td.ldf = nb;
            td.frows = nb;
          }
          tb.add(td);
        } else {
          tb.flush();
          size_t mark = ar.off;
          std::vector<Prob> sub(1);
          sub[0] = Prob{w, nullptr, 0, D, p.ldx, p.info, nullptr, nullptr, p.col0 + j};
          if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
          run_fwd(c, sub, kTileMax, ar);
          trtri_big(c, D, p.ldx, p.dinv + slot, nb, w, ar);
          ar.off = mark;
        }
      }
      tb.flush();
    }
    // f3 (both parts) of this block column and its panel split, and the previous step's panel
    // solve on the side stream (it reads the split inverse, overwritten below)
    if (s >= 1) c.wait(c.h->ev_near);
    if (s == 0) split_panel(0, false);  // later panels are split on the side stream (below)
    {  // D^{-1} for the panel solve
      if (fx) {
        FSplitBatch sb(c, true);
        for (auto &p : P) {
          if (j >= p.n) continue;
          const int w = std::min(p.n, j + nb) - j;
          if (p.n - j - w <= 0 || (w <= kTileMax && nb <= kTileMax)) continue;  // the tile kernel wrote it
          sb.add(p.dinv + slot, nb, w, w, 0, fP4s(p, s), nb, nb, 0, 0, nb, nb, 0, 0, exP4s(p, s));
        }
      } else {
        SplitBatch sb(c);
        for (auto &p : P) {
          if (j >= p.n) continue;
          const int w = std::min(p.n, j + nb) - j;
          if (p.n - j - w <= 0 || (w <= kTileMax && nb <= kTileMax)) continue;  // the tile kernel wrote it
          sb.add(p.dinv + slot, nb, w, w, 0, 0, P4s(p, s), nb, nb, 0, 0, nb, nb, 0, 0, T);
        }
      }
    }
    // f4: C <- C tril(D)^{-T}.  The next diagonal block needs only the panel's top nb rows: those
    // are solved and split on the chain; the other rows on the side stream.
    const bool more = s + 1 < steps;
    auto f4 = [&](bool top, bool on_side) {
      MixedBatch mb(c, T, false, on_side, "f4", fx);
      for (auto &p : P) {
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        const int r0 = top ? 0 : (more ? nb : 0), r1 = top && more ? std::min(m, nb) : m;
        if (r1 <= r0) continue;
        double *Cb = p.X + (long long)(k + r0) * p.ldx + j;  // in place: the product reads only the split copies
        if (fx)
          mb.add(fop(p.mx.fP1, nb, p.n, p.mx.exP1, 0, r0), fop(fP4s(p, s), nb, nb, exP4s(p, s), 0, 0), r1 - r0, w, w,
                 nullptr, 0, Cb, p.ldx, 1.0, 0.0);
        else
          mb.add(mop(p.mx.P1, nb, p.n, T, 0, r0), mop(P4s(p, s), nb, nb, T, 0, 0), r1 - r0, w, w, nullptr, 0, Cb,
                 p.ldx, 1.0, 0.0);
      }
    };
    // the finished rows [j + row0, j + row1) of this block column join the split operand
    auto split_col = [&](bool top, bool on_side) {
      if (fx) {
        FSplitBatch sb(c, false, on_side);
        for (auto &p : P) {
          if (j >= p.n) continue;
          const int w = std::min(p.n, j + nb) - j;
          const int h0 = top ? 0 : (more ? std::min(p.n - j, w + nb) : 0);
          const int h1 = top && more ? std::min(p.n - j, w + nb) : p.n - j;
          if (h1 <= h0) continue;
          sb.add(p.X + (long long)j * p.ldx + j, p.ldx, p.n - j, w, 1, p.mx.fbig, (p.n + 63) / 64 * 64, p.n, j + h0,
                 j, h1 - h0, w, j, j, p.mx.exL);
        }
      } else {
        SplitBatch sb(c, on_side);
        for (auto &p : P) {
          if (j >= p.n) continue;
          const int w = std::min(p.n, j + nb) - j;
          const int h0 = top ? 0 : (more ? std::min(p.n - j, w + nb) : 0);
          const int h1 = top && more ? std::min(p.n - j, w + nb) : p.n - j;
          if (h1 <= h0) continue;
          sb.add(p.X + (long long)j * p.ldx + j, p.ldx, p.n - j, w, 1, 0, p.mx.big, p.mx.ldb, p.n, j + h0, j,
                 h1 - h0, w, j, j, T);
        }
      }
    };
    if (more) {
      c.fork();  // the side stream starts the panel's other rows as soon as D^{-1} is split
      f4(false, true);
      split_col(false, true);
    }
    f4(true, false);
    split_col(true, false);
    if (after) (*after)(s);
    if (s + 1 < steps) {
      // f1 of the next block column, new part (this block column), on the chain before the side
      // stream's work so that its CTAs take SMs first; after the old part on the side stream
      if (look_set[(s + 1) & 1]) c.wait(c.h->ev_look[(s + 1) & 1]);
      upd(s + 1, j, j + nb, false, true, false);
      // side stream: the next block column's new f3 part and its panel split, then block s + 2's
      // old parts
      c.fork();
      upd(s + 1, j, j + nb, true, false, true);
      split_panel(s + 1, true);
      c.record(c.h->ev_near);
      if (s + 2 < steps) {
        upd(s + 2, 0, j + nb, true, true, false);
        c.record(c.h->ev_look[(s + 2) & 1]);
        look_set[(s + 2) & 1] = true;
        upd(s + 2, 0, j + nb, true, false, true);
      }
    }
  }
}

// One block step of chol_blocked_fwd (Sec. 4.2), products in split BF16: p.L is the factor
// (its split `big` holds at least columns [0, j + nb)), p.X the sensitivity L_dot, whose finished
// columns go to `big2`; p.dinv's slot s holds the block's D^{-1}.
void sens_mixed_step(Ctx &c, std::vector<Prob> &P, int nb, int s, int T, Arena &ar) {
  c.fork();
  {  // g1: D_dot <- D_dot - tril(R_dot R^T + R R_dot^T) = D_dot - tril(P + P^T), P = R_dot R^T:
     // one product into T1, then the symmetric update (enqueued before the side stream's g3,
     // so that its CTAs take SMs first)
    {
      MixedBatch mb(c, T, false, false, "g1");
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int w = std::min(p.n, j + nb) - j;
        mb.add(mop(p.mx.big2, p.mx.ldb, p.n, T, 0, j), mop(p.mx.big, p.mx.ldb, p.n, T, 0, j), w, w, j, nullptr, 0,
               p.T1, nb, 1.0, 0.0);
      }
    }
    CopyBatch sym(c, true);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n || j == 0) continue;  // j = 0: no columns to the left, no product
      const int w = std::min(p.n, j + nb) - j;
      sym.add(p.T1, nb, p.X + (long long)j * p.ldx + j, p.ldx, w, w);
    }
  }
  for (int term = 0; term < 2; ++term) {  // g3 (side stream): C_dot <- C_dot - B_dot R^T - B R_dot^T
    MixedBatch mb(c, T, false, true, "g3");
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      double *Cd = p.X + (long long)k * p.ldx + j;
      void *a = term == 0 ? p.mx.big2 : p.mx.big, *b = term == 0 ? p.mx.big : p.mx.big2;
      mb.add(mop(a, p.mx.ldb, p.n, T, 0, k), mop(b, p.mx.ldb, p.n, T, 0, j), m, w, j, Cd, p.ldx, Cd, p.ldx, -1.0,
             1.0);
    }
  }
  {  // g2 as the products of Eq. symfwd (problems that use them)
    std::vector<DiagRev> v;
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n || !diag_symbolic(c, p, nb)) continue;
      const int w = std::min(p.n, j + nb) - j;
      v.push_back({p.L + (long long)j * p.ldl + j, p.ldl, p.X + (long long)j * p.ldx + j, p.ldx,
                   p.dinv + (size_t)s * nb * nb, p.T1, p.T2, w, nb});
    }
    if (!v.empty()) sens_diag_symbolic(c, v);
  }
  {  // g2: D_dot <- chol_unblocked_fwd(D, D_dot)   (FP64)
    TileBatch tb(c, T_SENS);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n || diag_symbolic(c, p, nb)) continue;
      const int w = std::min(p.n, j + nb) - j;
      const double *D = p.L + (long long)j * p.ldl + j;
      double *Dd = p.X + (long long)j * p.ldx + j;
      if (w <= kTileMax) {
        tb.add(tdesc(D, p.ldl, Dd, p.ldx, nullptr, 0, w));
      } else {
        tb.flush();
        size_t mark = ar.off;
        std::vector<Prob> sub(1);
        sub[0] = Prob{w, D, p.ldl, Dd, p.ldx, nullptr, nullptr, nullptr, 0};
        if (!bind_workspace(sub, kTileMax, ar)) { c.err = CD_ENOMEM; return; }
        run_sens(c, sub, kTileMax, ar);
        ar.off = mark;
      }
    }
  }
  c.join();
  {  // g4a: C_dot <- C_dot - C D_dot^T
    {
      SplitBatch sb(c);
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        if (m <= 0) continue;
        sb.add(p.X + (long long)j * p.ldx + j, p.ldx, w, w, 1, 0, p.mx.P4, nb, nb, 0, 0, nb, nb, 0, 0, T);
      }
    }
    MixedBatch mb(c, T, false, false, "g4a");
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      double *Cd = p.X + (long long)k * p.ldx + j;
      mb.add(mop(p.mx.big, p.mx.ldb, p.n, T, j, k), mop(p.mx.P4, nb, nb, T, 0, 0), m, w, w, Cd, p.ldx, Cd, p.ldx,
             -1.0, 1.0);
    }
  }
  {  // g4b: C_dot <- C_dot D^{-T}
    {
      SplitBatch sb(c);
      for (auto &p : P) {
        const int j = s * nb;
        if (j >= p.n) continue;
        const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
        if (m <= 0) continue;
        sb.add(p.X + (long long)k * p.ldx + j, p.ldx, m, w, 0, 0, p.mx.P1, nb, p.n, 0, 0, m, nb, 0, 0, T);
        sb.add(p.dinv + (size_t)s * nb * nb, nb, w, w, 0, 0, p.mx.P4, nb, nb, 0, 0, nb, nb, 0, 0, T);
      }
    }
    MixedBatch mb(c, T, false, false, "g4b");
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      double *Cb = p.X + (long long)k * p.ldx + j;  // in place: the product reads only the split copies
      mb.add(mop(p.mx.P1, nb, p.n, T, 0, 0), mop(p.mx.P4, nb, nb, T, 0, 0), m, w, w, nullptr, 0, Cb, p.ldx, 1.0,
             0.0);
    }
  }
  {
    SplitBatch sb(c);
    for (auto &p : P) {
      const int j = s * nb;
      if (j >= p.n) continue;
      const int k = std::min(p.n, j + nb), w = k - j, m = p.n - k;
      sb.add(p.X + (long long)j * p.ldx + j, p.ldx, p.n - j, w, 1, 0, p.mx.big2, p.mx.ldb, p.n, j, j, p.n - j,
            w, j, j, T);
    }
  }
}

// chol_blocked_fwd (Sec. 4.2), products in split BF16: L is split once into
// `big`, the finished columns of L_dot into `big2`.
void run_sens_mixed(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  precompute_dinv(c, P, nb, false, ar);
  {
    SplitBatch sb(c);
    for (auto &p : P)
      sb.add(p.L, p.ldl, p.n, p.n, 1, 0, p.mx.big, p.mx.ldb, p.n, 0, 0, p.n, (int)p.mx.ldb, 0, 0, p.mx.T);
  }
  const int T = P.empty() ? 2 : P[0].mx.T;
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  for (int s = 0; s < steps && c.err == CD_OK; ++s) sens_mixed_step(c, P, nb, s, T, ar);
}

// chol_blocked and chol_blocked_fwd (Sec. 4.1 takes both in one loop), products in split BF16
// or, for the factor, fixed-point slices.  The factorisation runs as in run_fwd_mixed, bound by
// its diagonal chain; each sensitivity step runs one block column behind it on a second chain
// and bulk stream (crit2, side2), started by events recorded once the factor's block column
// is final on both of the factorisation's streams, so that it fills the SMs the chain leaves
// idle.  The sensitivity steps take every block's D^{-1} from its slot of p.dinv, their own
// scratch (P2/P3 for the panel and D^{-1} splits of the three-term split, T1/T2, partials) and,
// under fixed4, their own three-term split of each finished block column of L (in `big`).
void run_dual_mixed(Ctx &c, std::vector<Prob> &P, int nb, Arena &ar) {
  const bool fx = c.opt->prec == CD_MIXED_FIXED4;
  const int T = P.empty() ? 2 : P[0].mx.T;  // the derivative products' split
  int nmax = 0;
  for (auto &p : P) nmax = std::max(nmax, p.n);
  const int steps = nblocks(nmax, nb);
  std::vector<Prob> S = P;  // the sensitivity pass's view: L = the factor being formed, X = L_dot
  for (auto &q : S) {
    q.L = q.X;
    q.ldl = q.ldx;
    q.X = q.Xd;
    q.ldx = q.ldxd;
    q.Xd = nullptr;
    if (!fx) {  // the factorisation splits its panel and D^{-1} into P1 / P4
      q.mx.P1 = q.mx.P2;
      q.mx.P4 = q.mx.P3;
    }
  }
  auto split_L = [&](Ctx &cc, int s) {  // fixed4: the three-term split of L's block column s
    if (!fx) return;                     // (the three-term factorisation writes it itself)
    SplitBatch sb(cc);
    for (auto &q : S) {
      const int j = s * nb;
      if (j >= q.n) continue;
      const int w = std::min(q.n, j + nb) - j;
      sb.add(q.L + (long long)j * q.ldl + j, q.ldl, q.n - j, w, 1, 0, q.mx.big, q.mx.ldb, q.n, j, j, q.n - j, w, j,
             j, T);
    }
  };
  cd_handle *h = c.h;
  if (nb > kTileMax || !h->crit2 || !h->side2 || !c.part3) {
    // wide blocks recurse through the shared arena: the two passes one after the other
    run_fwd_mixed(c, P, nb, ar, nullptr, true);
    c.join();
    for (int s = 0; s < steps && c.err == CD_OK; ++s) {
      split_L(c, s);
      sens_mixed_step(c, S, nb, s, T, ar);
    }
    return;
  }
  Ctx sc = c;
  sc.s = h->crit2;
  sc.side = h->side2;
  sc.part = c.part3;
  sc.part_cap = c.part3_cap;
  sc.part2 = c.part4;
  sc.part2_cap = c.part3_cap;
  c.cuda(cudaEventRecord(h->ev_start2, c.s));
  c.cuda(cudaStreamWaitEvent(sc.s, h->ev_start2, 0));
  const std::function<void(int)> after = [&](int s) {
    // block column s of L is final: its top rows on the chain, the rest on the side stream
    c.cuda(cudaEventRecord(h->ev_colA, c.s));
    c.cuda(cudaStreamWaitEvent(sc.s, h->ev_colA, 0));
    if (c.side) {
      c.cuda(cudaEventRecord(h->ev_colB, c.side));
      c.cuda(cudaStreamWaitEvent(sc.s, h->ev_colB, 0));
    }
    if (sc.err != CD_OK) return;
    split_L(sc, s);
    sens_mixed_step(sc, S, nb, s, T, ar);
  };
  run_fwd_mixed(c, P, nb, ar, &after, true);
  sc.join();
  c.cuda(cudaEventRecord(h->ev_start2, sc.s));
  c.cuda(cudaStreamWaitEvent(c.s, h->ev_start2, 0));
  if (c.err == CD_OK && sc.err != CD_OK) c.err = sc.err;
}

enum Op { OP_FWD, OP_REV, OP_SENS, OP_DUAL };

// Split-K partial region of one stream: 64 MB, or for the split-BF16 path
// enough for its longest products (nb x n outputs, K up to n, FP32
// accumulation over at most kMixMaxChunk of K) so that no split is capped.
size_t part_bytes(int nmax, int nb, bool mixed) {
  size_t b = kPartBytes;
  if (mixed) {
    const size_t need = sizeof(double) * (size_t)nb * nmax * (size_t)((nmax + kMixMaxChunk - 1) / kMixMaxChunk);
    b = std::max(b, need);
  }
  return align_up(b);
}

size_t need_bytes(const int *n, int batch, int nb, bool mixed = false, bool dual = false) {
  int nmax = 0;
  for (int i = 0; i < batch; ++i) nmax = std::max(nmax, n[i]);
  // (the one-loop pass runs its sensitivity steps on two more streams, with partials of their own)
  size_t b = (dual ? 4 : 2) * part_bytes(nmax, nb, mixed) + recursion_bytes(nb) + 4 * kAlign;
  for (int i = 0; i < batch; ++i) b += prob_bytes(n[i], nb, dual) + 2 * kAlign;
  return b;
}

// Grow the workspace in stream order: the old buffer is released after the
// work already enqueued on `s` (which every earlier call of this handle has
// joined back into) and the new one is usable by work enqueued after it, so
// growing never waits for the device.
int ensure_ws(cd_handle *h, size_t bytes, cudaStream_t s, bool headroom = true) {
  if (bytes <= h->ws_bytes) return CD_OK;
  if (h->ws) {
    cudaFreeAsync(h->ws, s);
    h->ws = nullptr;
    h->ws_bytes = 0;
  }
  if (headroom) bytes = bytes + bytes / 8;  // fewer regrowths for slowly growing batches
  if (cudaMallocAsync(&h->ws, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return CD_ENOMEM;
  }
  h->ws_bytes = bytes;
  return CD_OK;
}

int run(cd_handle *h, Op op, int batch, const int *n, const double *const *L, const long long *ldl,
        double *const *X, const long long *ldx, const cd_options *opt_in, void *stream, int *info,
        double *const *Xd = nullptr, const long long *ldxd = nullptr) {
  if (!h || batch < 0 || (batch > 0 && (!n || !X || !ldx))) return CD_EINVAL;
  if (op == OP_DUAL && batch > 0 && (!Xd || !ldxd)) return CD_EINVAL;
  cd_options opt;
  cd_options_default(&opt);
  if (opt_in) opt = *opt_in;
  if (opt.nb < 0 || opt.prec < CD_FP64 || opt.prec > CD_MIXED_FIXED4 || opt.out < CD_OUT_TRIL ||
      opt.out > CD_OUT_SYM || opt.diag < CD_DIAG_AUTO || opt.diag > CD_DIAG_SYMBOLIC || opt.uplo < CD_LOWER ||
      opt.uplo > CD_UPPER)
    return CD_EINVAL;
  int nmax = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 0 || ldx[b] < std::max(1, n[b])) return CD_EINVAL;
    if (n[b] > 0 && !X[b]) return CD_EINVAL;
    if (op == OP_REV || op == OP_SENS) {
      if (!L || !ldl) return CD_EINVAL;
      if (n[b] > 0 && (!L[b] || ldl[b] < n[b])) return CD_EINVAL;
    }
    if (op == OP_DUAL) {
      if (ldxd[b] < std::max(1, n[b])) return CD_EINVAL;
      if (n[b] > 0 && (!Xd[b] || Xd[b] == X[b])) return CD_EINVAL;
    }
    nmax = std::max(nmax, n[b]);
  }
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool factor = op == OP_FWD || op == OP_DUAL;
  if (factor && info && batch > 0) {
    if (cudaMemsetAsync(info, 0, sizeof(int) * batch, s) != cudaSuccess) return CD_ECUDA;
  }
  if (nmax == 0) return CD_OK;
  const int nb = pick_nb(nmax, &opt, factor);
  size_t need = need_bytes(n, batch, nb, opt.prec != CD_FP64, op == OP_DUAL);
  if (opt.prec != CD_FP64)
    for (int b = 0; b < batch; ++b)
      need += mix_bytes(n[b], nb, mix_terms(opt.prec), op == OP_SENS || op == OP_DUAL,
                        opt.prec == CD_MIXED_FIXED4 && factor, op == OP_REV);
  const bool upper = opt.uplo == CD_UPPER;
  const int narr = 1 + (factor ? 0 : 1) + (op == OP_DUAL ? 1 : 0);  // matrices per problem
  if (upper)
    for (int b = 0; b < batch; ++b) need += narr * (align_up(sizeof(double) * (size_t)n[b] * n[b]) + kAlign);
  int rc = ensure_ws(h, need, s);
  if (rc) return rc;

  Arena ar;
  ar.base = (char *)h->ws;
  ar.cap = h->ws_bytes;
  Ctx c{h, s, &opt, nullptr, 0, h->gemm_slots};
  const size_t pb = part_bytes(nmax, nb, opt.prec != CD_FP64);
  c.part = (double *)ar.take(pb);
  c.part_cap = pb / sizeof(double);
  c.side = h->side;
  c.part2 = (double *)ar.take(pb);
  c.part2_cap = pb / sizeof(double);
  if (op == OP_DUAL) {
    c.part3 = (double *)ar.take(pb);
    c.part4 = (double *)ar.take(pb);
    c.part3_cap = pb / sizeof(double);
  }
  // CD_UPPER: each operand's upper triangle, transposed, in a workspace copy
  // (ld n) on which the lower-triangle algorithms run; results go back below.
  struct Copy {
    double *user, *work;
    long long ld;
    int n;
    bool out;
  };
  std::vector<Copy> copies;
  auto staged = [&](const double *user, long long ld, int nn, bool out) -> double * {
    double *w = (double *)ar.take(sizeof(double) * (size_t)nn * nn);
    if (!w) return nullptr;
    copies.push_back({const_cast<double *>(user), w, ld, nn, out});
    c.launch("transpose_f64", 0.0, 16.0 * 0.5 * nn * (nn + 1.0),
             [&] { return launch_transpose(user, ld, w, nn, nn, 0, s); });
    return w;
  };
  std::vector<Prob> P;
  P.reserve(batch);
  for (int b = 0; b < batch; ++b) {
    if (n[b] == 0) continue;
    Prob p{n[b], factor ? nullptr : L[b], factor ? 0 : ldl[b], X[b], ldx[b], info ? info + b : nullptr,
           nullptr, nullptr, 0};
    if (op == OP_DUAL) {
      p.Xd = Xd[b];
      p.ldxd = ldxd[b];
    }
    if (upper) {
      p.X = staged(X[b], ldx[b], n[b], true);
      p.ldx = n[b];
      if (!factor) {
        p.L = staged(L[b], ldl[b], n[b], false);
        p.ldl = n[b];
      }
      if (op == OP_DUAL) {
        p.Xd = staged(Xd[b], ldxd[b], n[b], true);
        p.ldxd = n[b];
      }
      if (!p.X || (!factor && !p.L) || (op == OP_DUAL && !p.Xd)) return CD_ENOMEM;
    }
    P.push_back(p);
  }
  if (!bind_workspace(P, nb, ar)) return CD_ENOMEM;
  const bool mixed = opt.prec != CD_FP64;
  const bool fixed = opt.prec == CD_MIXED_FIXED4 && factor;
  if (mixed && mixed_init() != CD_OK) return CD_ECUDA;  // per device, once
  if (fixed && fixed_init() != CD_OK) return CD_ECUDA;
  if (mixed && !bind_mixed(P, nb, mix_terms(opt.prec), op == OP_SENS || op == OP_DUAL, ar, fixed, op == OP_REV))
    return CD_ENOMEM;
  // The step loops issue the diagonal chain on the high-priority stream (its
  // CTAs are scheduled first when SM slots free up) and the independent bulk
  // GEMM of each step on the side stream; both start after, and the caller's
  // stream resumes after, all of it.
  if (h->crit) {
    c.cuda(cudaEventRecord(h->ev_in, s));
    c.cuda(cudaStreamWaitEvent(h->crit, h->ev_in, 0));
    c.s = h->crit;
  }
  switch (op) {
    case OP_FWD: mixed ? run_fwd_mixed(c, P, nb, ar) : run_fwd(c, P, nb, ar); break;
    case OP_REV: mixed ? run_rev_mixed(c, P, nb, ar) : run_rev(c, P, nb, ar); break;
    case OP_SENS: mixed ? run_sens_mixed(c, P, nb, ar) : run_sens(c, P, nb, ar); break;
    case OP_DUAL: mixed ? run_dual_mixed(c, P, nb, ar) : run_dual(c, P, nb, ar); break;
  }
  if (h->crit) {
    c.join();
    c.cuda(cudaEventRecord(h->ev_out, h->crit));
    c.cuda(cudaStreamWaitEvent(s, h->ev_out, 0));
    c.s = s;
  }
  if (c.err) return c.err;
  const bool sym = op == OP_REV && opt.out == CD_OUT_SYM;
  if (sym)
    for (auto &p : P)
      c.launch("mirror_f64", 0.0, 8.0 * p.n * (p.n - 1.0),
               [&] { return launch_mirror_lower(p.X, p.ldx, p.n, s); });
  for (auto &cp : copies)  // CD_UPPER: results back to the upper triangles (every element for CD_OUT_SYM)
    if (cp.out)
      c.launch("transpose_f64", 0.0, 16.0 * 0.5 * cp.n * (cp.n + 1.0),
               [&] { return launch_transpose(cp.work, cp.n, cp.user, cp.ld, cp.n, sym ? 2 : 1, s); });
  return c.err;
}

bool g_init_done = false;

}  // namespace

namespace cd {

// Workspace bytes the reverse pass needs for one problem of size n with block
// size nb when nb <= kTileMax (inverse blocks and the solved panel; split-K
// partial sums use whatever is left and are optional).
size_t rev_scratch_need(int n, int nb) { return prob_bytes(n, nb) + 2 * kAlign; }

// The reverse pass of one problem with every scratch word taken from the
// given device block instead of the handle's workspace.  Used by
// cd_chol_rev_noalloc; performs no allocation.  nb must be <= kTileMax.
int rev_in_scratch(int n, const double *L, long long ldl, double *Abar, long long lda, int nb, int out,
                   void *scratch, size_t scratch_bytes, int num_sms, cudaStream_t s) {
  cd_handle hh;
  memset(&hh, 0, sizeof(hh));
  cudaGetDevice(&hh.device);
  hh.num_sms = num_sms;
  // the same partition as cd_create's handle (occupancy queries: no allocation)
  hh.gemm_slots = gemm_ctas_per_sm(64) * num_sms;
  hh.gemm_slots_small = gemm_ctas_per_sm(32) * num_sms;
  Arena ar;
  ar.base = (char *)scratch;
  ar.cap = scratch_bytes;
  cd_options opt;
  cd_options_default(&opt);
  opt.nb = nb;
  opt.out = out;
  opt.diag = CD_DIAG_LEVEL2;
  std::vector<Prob> P(1);
  P[0] = Prob{n, L, ldl, Abar, lda, nullptr, nullptr, nullptr, 0};
  if (!bind_workspace(P, nb, ar)) return CD_EINVAL;
  Ctx c{&hh, s, &opt, nullptr, 0, hh.gemm_slots};
  const size_t left = ar.cap > align_up(ar.off) ? ar.cap - align_up(ar.off) : 0;
  c.part_cap = left / sizeof(double);
  c.part = c.part_cap ? (double *)ar.take(c.part_cap * sizeof(double)) : nullptr;
  if (!c.part) c.part_cap = 0;
  run_rev(c, P, nb, ar);
  if (c.err) return c.err;
  if (out == CD_OUT_SYM) c.check(launch_mirror_lower(Abar, lda, n, s));
  return c.err;
}

}  // namespace cd

extern "C" {

const char *cd_version(void) { return "libcholdiff 0.1 (sm_103a)"; }

void cd_options_default(cd_options *opt) {
  if (!opt) return;
  opt->nb = 0;
  opt->prec = CD_FP64;
  opt->out = CD_OUT_TRIL;
  opt->diag = CD_DIAG_AUTO;
  opt->uplo = CD_LOWER;
  opt->spin_limit = 0;
}

int cd_create(cd_handle **h, int device) {
  if (!h) return CD_EINVAL;
  *h = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess) {
    cudaGetLastError();
    return CD_ECUDA;
  }
  if (device < 0 || device >= count) return CD_EINVAL;
  DeviceGuard guard(device);
  cd_handle *x = (cd_handle *)calloc(1, sizeof(cd_handle));
  if (!x) return CD_ENOMEM;
  x->device = device;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    free(x);
    return CD_ECUDA;
  }
  x->num_sms = prop.multiProcessorCount;
  x->smem_optin = prop.sharedMemPerBlockOptin;
  if (tile_kernels_init() != cudaSuccess) {
    free(x);
    return CD_ECUDA;
  }
  mixed_init();  // on failure only the CD_MIXED_* paths are unavailable
  fixed_init();
  g_init_done = true;
  if (cudaMalloc(&x->dev_err, sizeof(int)) != cudaSuccess || cudaMemset(x->dev_err, 0, sizeof(int)) != cudaSuccess) {
    free(x);
    return CD_ECUDA;
  }
  x->gemm_slots = gemm_ctas_per_sm(64) * x->num_sms;
  x->gemm_slots_small = gemm_ctas_per_sm(32) * x->num_sms;
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&x->side, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaStreamCreateWithPriority(&x->crit, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaStreamCreateWithPriority(&x->side2, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaStreamCreateWithPriority(&x->crit2, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_colA, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_colB, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_start2, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_mid, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_look[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_look[1], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&x->ev_near, cudaEventDisableTiming) != cudaSuccess) {
    cudaFree(x->dev_err);
    free(x);
    return CD_ECUDA;
  }
  *h = x;
  return CD_OK;
}

int cd_destroy(cd_handle *h) {
  if (!h) return CD_OK;
  DeviceGuard guard(h->device);
  delete (Profiler *)h->prof;
  if (h->ws) cudaFree(h->ws);
  if (h->dev_err) cudaFree(h->dev_err);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->crit) cudaStreamDestroy(h->crit);
  if (h->side2) cudaStreamDestroy(h->side2);
  if (h->crit2) cudaStreamDestroy(h->crit2);
  if (h->ev_colA) cudaEventDestroy(h->ev_colA);
  if (h->ev_colB) cudaEventDestroy(h->ev_colB);
  if (h->ev_start2) cudaEventDestroy(h->ev_start2);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  for (int q = 0; q < 2; ++q)
    if (h->ev_look[q]) cudaEventDestroy(h->ev_look[q]);
  if (h->ev_near) cudaEventDestroy(h->ev_near);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->ev_mid) cudaEventDestroy(h->ev_mid);
  free(h);
  return CD_OK;
}

int cd_workspace_size(const cd_handle *h, int n_max, const cd_options *opt, size_t *bytes) {
  if (!h || !bytes || n_max < 0) return CD_EINVAL;
  const int nb = pick_nb(n_max, opt);
  *bytes = need_bytes(&n_max, 1, nb, opt && opt->prec != CD_FP64, true) +
           ((opt && opt->prec != CD_FP64) ? mix_bytes(n_max, nb, mix_terms(opt->prec), true,
                                                      opt->prec == CD_MIXED_FIXED4, true) : 0) +
           ((opt && opt->uplo == CD_UPPER) ? 3 * (align_up(sizeof(double) * (size_t)n_max * n_max) + kAlign) : 0);
  return CD_OK;
}

int cd_workspace_size_batched(const cd_handle *h, int batch, const int *n, const cd_options *opt, size_t *bytes) {
  if (!h || !bytes || batch < 0 || (batch > 0 && !n)) return CD_EINVAL;
  int nmax = 0;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 0) return CD_EINVAL;
    nmax = std::max(nmax, n[b]);
  }
  const int nb = pick_nb(nmax, opt);
  const bool mixed = opt && opt->prec != CD_FP64;
  size_t need = need_bytes(n, batch, nb, mixed, true);
  for (int b = 0; b < batch; ++b) {
    if (mixed) need += mix_bytes(n[b], nb, mix_terms(opt->prec), true, opt->prec == CD_MIXED_FIXED4, true);
    if (opt && opt->uplo == CD_UPPER) need += 3 * (align_up(sizeof(double) * (size_t)n[b] * n[b]) + kAlign);
  }
  *bytes = need;
  return CD_OK;
}

int cd_workspace_bytes(const cd_handle *h, size_t *bytes) {
  if (!h || !bytes) return CD_EINVAL;
  *bytes = h->ws_bytes;
  return CD_OK;
}

int cd_reserve(cd_handle *h, size_t bytes) {
  if (!h) return CD_EINVAL;
  DeviceGuard guard(h->device);
  const int rc = ensure_ws(h, bytes, nullptr, false);  // exactly what the caller reserves
  if (rc == CD_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) return CD_ECUDA;
  return rc;
}

int cd_chol_fwd(cd_handle *h, int n, double *A, long long lda, const cd_options *opt, void *stream, int *info) {
  double *X[1] = {A};
  long long ld[1] = {lda};
  return run(h, OP_FWD, 1, &n, nullptr, nullptr, X, ld, opt, stream, info);
}

int cd_chol_rev(cd_handle *h, int n, const double *L, long long ldl, double *Abar, long long lda,
                const cd_options *opt, void *stream) {
  const double *Lp[1] = {L};
  long long ll[1] = {ldl};
  double *X[1] = {Abar};
  long long ld[1] = {lda};
  return run(h, OP_REV, 1, &n, Lp, ll, X, ld, opt, stream, nullptr);
}

int cd_chol_fwd_sens(cd_handle *h, int n, const double *L, long long ldl, double *Adot, long long lda,
                     const cd_options *opt, void *stream) {
  const double *Lp[1] = {L};
  long long ll[1] = {ldl};
  double *X[1] = {Adot};
  long long ld[1] = {lda};
  return run(h, OP_SENS, 1, &n, Lp, ll, X, ld, opt, stream, nullptr);
}

int cd_chol_fwd_batched(cd_handle *h, int batch, const int *n, double *const *A, const long long *lda,
                        const cd_options *opt, void *stream, int *info) {
  return run(h, OP_FWD, batch, n, nullptr, nullptr, A, lda, opt, stream, info);
}

int cd_chol_rev_batched(cd_handle *h, int batch, const int *n, const double *const *L, const long long *ldl,
                        double *const *Abar, const long long *lda, const cd_options *opt, void *stream) {
  return run(h, OP_REV, batch, n, L, ldl, Abar, lda, opt, stream, nullptr);
}

int cd_chol_fwd_sens_batched(cd_handle *h, int batch, const int *n, const double *const *L, const long long *ldl,
                             double *const *Adot, const long long *lda, const cd_options *opt, void *stream) {
  return run(h, OP_SENS, batch, n, L, ldl, Adot, lda, opt, stream, nullptr);
}

int cd_chol_fwd_and_sens(cd_handle *h, int n, double *A, long long lda, double *Adot, long long ldadot,
                         const cd_options *opt, void *stream, int *info) {
  double *X[1] = {A}, *Xd[1] = {Adot};
  long long ld[1] = {lda}, ldd[1] = {ldadot};
  return run(h, OP_DUAL, 1, &n, nullptr, nullptr, X, ld, opt, stream, info, Xd, ldd);
}

int cd_chol_fwd_and_sens_batched(cd_handle *h, int batch, const int *n, double *const *A, const long long *lda,
                                 double *const *Adot, const long long *ldadot, const cd_options *opt, void *stream,
                                 int *info) {
  return run(h, OP_DUAL, batch, n, nullptr, nullptr, A, lda, opt, stream, info, Adot, ldadot);
}

int cd_chol_jacobian(cd_handle *h, int n, const double *L, long long ldl, double *J, void *stream) {
  if (!h || n < 0 || (n > 0 && (!L || !J || ldl < n))) return CD_EINVAL;
  if (n == 0) return CD_OK;
  DeviceGuard guard(h->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t need = align_up(sizeof(double) * (size_t)n * n) + align_up(sizeof(double) * (size_t)n * n * n) +
                      align_up(sizeof(double) * (size_t)n * n) + 8 * kAlign;  // L^{-1}, S, the inverse's scratch
  int rc = ensure_ws(h, need, s);
  if (rc) return rc;
  Arena ar;
  ar.base = (char *)h->ws;
  ar.cap = h->ws_bytes;
  cd_options opt;
  cd_options_default(&opt);
  Ctx c{h, s, &opt, nullptr, 0, h->gemm_slots};
  double *Li = (double *)ar.take(sizeof(double) * (size_t)n * n);
  double *S = (double *)ar.take(sizeof(double) * (size_t)n * n * n);
  if (!Li || !S) return CD_ENOMEM;
  trtri_big(c, L, ldl, Li, n, n, ar);  // L^{-1}, full storage, zeros above the diagonal
  if (c.err) return c.err;
  const double n4 = (double)n * n * n * n;
  c.launch("jacobian", 4.0 * n4, 8.0 * n4, [&] { return launch_jacobian(n, L, ldl, Li, n, S, J, s); });
  return c.err;
}

int cd_debug_fp64_helpers(cd_handle *h, int n, const double *x, double *recip, double *sq, double *rsq,
                          void *stream) {
  if (!h || n < 0 || (n > 0 && (!x || !recip || !sq || !rsq))) return CD_EINVAL;
  DeviceGuard guard(h->device);
  const cudaError_t e = launch_fp64_helpers(n, x, recip, sq, rsq, (cudaStream_t)stream);
  ++h->launches;
  return e == cudaSuccess ? CD_OK : CD_ECUDA;
}

int cd_debug_fp64_probe(cd_handle *h, int kind, long long iters, void *stream, double *flops) {
  if (!h || (kind != 0 && kind != 1) || iters < 1 || !flops) return CD_EINVAL;
  DeviceGuard guard(h->device);
  const cudaError_t e = launch_fp64_probe(kind, 4 * h->num_sms, iters, (cudaStream_t)stream, flops);
  ++h->launches;
  return e == cudaSuccess ? CD_OK : CD_ECUDA;
}

int cd_set_priorities(cd_handle *h, int chain_priority, int bulk_priority) {
  if (!h) return CD_EINVAL;
  DeviceGuard guard(h->device);
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  auto clamp = [&](int p) { return std::min(lo, std::max(hi, p)); };
  if (cudaDeviceSynchronize() != cudaSuccess) return CD_ECUDA;
  cudaStream_t st[4] = {nullptr, nullptr, nullptr, nullptr};  // crit, side, crit2, side2
  for (int q = 0; q < 4; ++q)
    if (cudaStreamCreateWithPriority(&st[q], cudaStreamNonBlocking, clamp(q % 2 ? bulk_priority : chain_priority)) !=
        cudaSuccess) {
      for (int r = 0; r < q; ++r) cudaStreamDestroy(st[r]);
      return CD_ECUDA;
    }
  cudaStreamDestroy(h->crit);
  cudaStreamDestroy(h->side);
  cudaStreamDestroy(h->crit2);
  cudaStreamDestroy(h->side2);
  h->crit = st[0];
  h->side = st[1];
  h->crit2 = st[2];
  h->side2 = st[3];
  return CD_OK;
}

int cd_mixed_gemm_debug(cd_handle *h, int M, int N, int K, const double *A, long long lda, const double *B,
                        long long ldb, double *C, long long ldc, int prec, int lower, void *stream) {
  if (!h || M < 0 || N < 0 || K < 1 ||
      (prec != CD_MIXED_BF16X3 && prec != CD_MIXED_BF16X6 && prec != CD_MIXED_FIXED4) || (lower && M != N))
    return CD_EINVAL;
  if (M == 0 || N == 0) return CD_OK;
  if (!A || !B || !C || lda < K || ldb < K || ldc < N) return CD_EINVAL;
  DeviceGuard guard(h->device);
  const bool fx = prec == CD_MIXED_FIXED4;
  if (mixed_init() != CD_OK || (fx && fixed_init() != CD_OK)) return CD_EINVAL;
  const int T = fx ? kFixedSlices : mix_terms(prec);
  const long long kp = (K + 63) / 64 * 64;
  const size_t bytes = kPartBytes + 2 * (size_t)T * ((size_t)M * kp + (size_t)N * kp) +
                       sizeof(int) * ((size_t)M + N) + 6 * kAlign;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(h, bytes, s);
  if (rc) return rc;
  Arena ar;
  ar.base = (char *)h->ws;
  ar.cap = h->ws_bytes;
  cd_options opt;
  cd_options_default(&opt);
  opt.prec = prec;
  Ctx c{h, s, &opt, nullptr, 0, h->gemm_slots};
  c.part = (double *)ar.take(kPartBytes);
  c.part_cap = kPartBytes / sizeof(double);
  void *As = ar.take(2 * (size_t)T * M * kp);
  void *Bs = ar.take(2 * (size_t)T * N * kp);
  int *ea = (int *)ar.take(sizeof(int) * M);
  int *eb = (int *)ar.take(sizeof(int) * N);
  if (!As || !Bs || !ea || !eb) return CD_ENOMEM;
  if (fx) {
    FSplitBatch sb(c, true);
    sb.add(A, lda, M, K, 0, As, kp, M, 0, 0, M, (int)kp, 0, 0, ea);
    sb.add(B, ldb, N, K, 0, Bs, kp, N, 0, 0, N, (int)kp, 0, 0, eb);
  } else {
    split(c, s, A, lda, M, K, 0, 0, As, kp, M, 0, 0, M, (int)kp, 0, 0, T);
    split(c, s, B, ldb, N, K, 0, 0, Bs, kp, N, 0, 0, N, (int)kp, 0, 0, T);
  }
  {
    MixedBatch mb(c, T, lower != 0, false, nullptr, fx);
    if (fx)
      mb.add(fop(As, kp, M, ea, 0, 0), fop(Bs, kp, N, eb, 0, 0), M, N, K, nullptr, 0, C, ldc, 1.0, 0.0);
    else
      mb.add(mop(As, kp, M, T, 0, 0), mop(Bs, kp, N, T, 0, 0), M, N, K, nullptr, 0, C, ldc, 1.0, 0.0);
  }
  return c.err;
}

int cd_debug_wait_timeout(cd_handle *h, void *stream) {
  if (!h) return CD_EINVAL;
  DeviceGuard guard(h->device);
  if (mixed_init() != CD_OK) return CD_EINVAL;
  const int T = 2, K = 64, M = 64;
  const size_t bytes = 2 * (size_t)T * 2 * M * K + sizeof(double) * M * M + 4 * kAlign;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = ensure_ws(h, bytes, s);
  if (rc) return rc;
  Arena ar;
  ar.base = (char *)h->ws;
  ar.cap = h->ws_bytes;
  void *As = ar.take(2 * (size_t)T * M * K);
  double *C = (double *)ar.take(sizeof(double) * M * M);
  if (!As || !C) return CD_ENOMEM;
  if (cudaMemsetAsync(As, 0, 2 * (size_t)T * M * K, s) != cudaSuccess) return CD_ECUDA;
  MProblem P;
  memset(&P, 0, sizeof(P));
  P.A = mop(As, K, M, T, 0, 0);
  P.B = P.A;
  P.M = P.N = M;
  P.K = K;
  P.Cout = C;
  P.ldcout = M;
  P.alpha = 1.0;
  P.splits = 1;
  P.kchunk = K;
  int l = 0;
  const cudaError_t e = mixed_gemm_launch(&P, 1, T, false, h->dev_err, s, &l, 16);
  h->launches += l;
  return e == cudaSuccess ? CD_OK : CD_ECUDA;
}

int cd_get_last_device_error(cd_handle *h, int *code) {
  if (!h || !code) return CD_EINVAL;
  DeviceGuard guard(h->device);
  int v = 0;
  if (cudaMemcpy(&v, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CD_ECUDA;
  if (cudaMemset(h->dev_err, 0, sizeof(int)) != cudaSuccess) return CD_ECUDA;
  *code = v;
  return CD_OK;
}

long long cd_launch_count(const cd_handle *h) { return h ? h->launches : 0; }

int cd_profile_enable(cd_handle *h, int on) {
  if (!h) return CD_EINVAL;
  if (on && !h->prof) h->prof = new Profiler();
  h->prof_on = on ? 1 : 0;
  return CD_OK;
}

int cd_profile_read(cd_handle *h, cd_kernel_stat *out, int max, int *count) {
  if (!h || !count || (max > 0 && !out)) return CD_EINVAL;
  *count = 0;
  Profiler *pr = (Profiler *)h->prof;
  if (!pr) return CD_OK;
  DeviceGuard guard(h->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return CD_ECUDA;
  std::vector<cd_kernel_stat> agg(pr->names.size());
  for (size_t i = 0; i < agg.size(); ++i) {
    memset(&agg[i], 0, sizeof(cd_kernel_stat));
    snprintf(agg[i].name, sizeof(agg[i].name), "%s", pr->names[i].c_str());
  }
  int rc = CD_OK;
  for (auto &r : pr->recs) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) rc = CD_ECUDA;
    cd_kernel_stat &a = agg[r.kind];
    a.launches += 1;
    a.ms += ms;
    a.flops += r.flops;
    a.bytes += r.bytes;
    pr->pool.push_back(r.e0);
    pr->pool.push_back(r.e1);
  }
  pr->recs.clear();
  std::sort(agg.begin(), agg.end(), [](const cd_kernel_stat &a, const cd_kernel_stat &b) { return a.ms > b.ms; });
  int k = 0;
  for (auto &a : agg)
    if (a.launches > 0 && k < max) out[k++] = a;
  *count = k;
  return rc;
}

int cd_profile_timeline(cd_handle *h, cd_launch_rec *out, int max, int *count) {
  if (!h || !count || (max > 0 && !out)) return CD_EINVAL;
  *count = 0;
  Profiler *pr = (Profiler *)h->prof;
  if (!pr || pr->recs.empty()) return CD_OK;
  DeviceGuard guard(h->device);
  if (cudaDeviceSynchronize() != cudaSuccess) return CD_ECUDA;
  const cudaEvent_t t0 = pr->recs[0].e0;
  int k = 0;
  for (auto &r : pr->recs) {
    if (k >= max) break;
    cd_launch_rec &o = out[k++];
    memset(&o, 0, sizeof(o));
    snprintf(o.name, sizeof(o.name), "%s", pr->names[r.kind].c_str());
    o.stream = r.side;
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, t0, r.e0) != cudaSuccess || cudaEventElapsedTime(&b, t0, r.e1) != cudaSuccess)
      return CD_ECUDA;
    o.start_ms = a;
    o.end_ms = b;
  }
  *count = k;
  return CD_OK;
}

}  // extern "C"
