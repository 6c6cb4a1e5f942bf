// Host-only check (no GPU needed) that the ensemble kernel's shared-memory
// carve and the host's size formula agree, for both samplers and both
// precisions, and that the launch shapes the host picks fit the device limit
// and hold the SVD working matrix they promise. Prints "ok <cases>" or the
// first mismatch and exits non-zero.
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "../paper_2604_13144_gb300/csrc/ensemble.cuh"
#include "../paper_2604_13144_gb300/csrc/host_plan.h"

using namespace tepai;

static bool aligned(const void* p, const void* base, size_t al) {
  return ((reinterpret_cast<uintptr_t>(p) - reinterpret_cast<uintptr_t>(base)) % al) == 0;
}

int main() {
  const size_t kOptin = 232448;      // 227 KB of dynamic shared memory per CTA on GB300
  const size_t kSmPerSm = 233472;    // 228 KB per SM
  static unsigned char pool[1 << 21];
  unsigned char* base = pool + (128 - reinterpret_cast<uintptr_t>(pool) % 128) % 128;
  long cases = 0;
  const int ns[] = {2, 3, 5, 8, 16, 33, 64, 100, 257, 1024};
  const int caps[] = {1, 2, 8, 16, 33, 64, 100, 128, 256};
  for (int n : ns)
    for (int periodic = 0; periodic < 2; ++periodic)
      for (int variant = 0; variant < 4; ++variant)
        for (int cap : caps)
          for (int csize : {8, 16}) {
            const int nb = periodic ? n : n - 1;
            KArgs a{};
            a.n = n; a.L = n + 3 * nb; a.variant = variant; a.chi_cap = cap;
            const SmemLayout s = carve_smem(base, a, csize);
            const int nclk = variant == 3 ? a.L : 0;
            const size_t fixed = smem_fixed_bytes(n, a.L, nclk, cap, csize);
            const size_t off = static_cast<size_t>(static_cast<unsigned char*>(s.x) - base);
            bool ok = off == fixed && aligned(s.x, base, 128) && aligned(s.tnext, base, 8) &&
                      aligned(s.tcnt, base, 4) && aligned(s.red, base, 8) && aligned(s.mbar, base, 8) &&
                      aligned(s.wn, base, 8) && aligned(s.perm, base, 4) && aligned(s.zval, base, 8) &&
                      aligned(s.dbuf, base, 8) && aligned(s.hh, base, 16);
            // regions in order, each at least as large as what the kernel indexes
            ok = ok && s.flags >= reinterpret_cast<unsigned char*>(s.dims + n + 1) &&
                 reinterpret_cast<unsigned char*>(s.tnext) >= s.flags + a.L &&
                 reinterpret_cast<unsigned char*>(s.tcnt) >= reinterpret_cast<unsigned char*>(s.tnext + nclk) &&
                 reinterpret_cast<unsigned char*>(s.red) >= reinterpret_cast<unsigned char*>(s.tcnt + nclk) &&
                 reinterpret_cast<unsigned char*>(s.mbar) >= reinterpret_cast<unsigned char*>(s.red + 64) &&
                 reinterpret_cast<unsigned char*>(s.wn) >= reinterpret_cast<unsigned char*>(s.mbar + 3) &&
                 reinterpret_cast<unsigned char*>(s.perm) >= reinterpret_cast<unsigned char*>(s.wn + 2 * cap) &&
                 reinterpret_cast<unsigned char*>(s.zval) >= reinterpret_cast<unsigned char*>(s.perm + 2 * cap) &&
                 reinterpret_cast<unsigned char*>(s.ibuf) >= reinterpret_cast<unsigned char*>(s.zval + n) &&
                 reinterpret_cast<unsigned char*>(s.dbuf) >= reinterpret_cast<unsigned char*>(s.ibuf + 16) &&
                 static_cast<unsigned char*>(s.hh) >= reinterpret_cast<unsigned char*>(s.dbuf + 16) &&
                 static_cast<unsigned char*>(s.x) >= static_cast<unsigned char*>(s.hh) + 3 * 2 * cap * csize;
            if (!ok) {
              std::printf("carve mismatch n=%d periodic=%d variant=%d cap=%d csize=%d off=%zu fixed=%zu\n", n,
                          periodic, variant, cap, csize, off, fixed);
              return 1;
            }
            // launch shapes: a simple occupancy model of the SM (shared memory with
            // 1 KB reserved per CTA, 64K registers at 128 per thread, 2048 threads)
            auto occ = [&](int block, size_t smem, int /*use_tc*/, int* per_sm) {
              int by_smem = static_cast<int>(kSmPerSm / (smem + 1024));
              int by_regs = 65536 / (block * 128);
              int by_thr = 2048 / block;
              int p = by_smem < by_regs ? by_smem : by_regs;
              *per_sm = p < by_thr ? p : by_thr;
              return cudaSuccess;
            };
            for (int lv = 0; lv <= 6; ++lv) {
              LaunchShape ls{};
              if (choose_launch_shape(n, a.L, nclk, cap, csize, static_cast<int>(kOptin), occ, ls, lv) !=
                  cudaSuccess)
                continue;
              if (fixed > kOptin) continue;   // such a problem is refused before launch
              const size_t xcap = ls.smem - fixed;
              bool good = ls.smem <= kOptin && ls.block >= 64 && ls.block <= 512 && ls.block % 32 == 0 &&
                          xcap >= static_cast<size_t>(ls.x_elems) * csize;
              if (ls.x_in_smem) good = good && ls.x_elems >= 4 * cap * cap;
              // staged: the Jacobi stages 4 bw m elements for a block width bw >= 1
              // (chosen from the buffer) and m <= 2 cap rows
              else good = good && ls.x_elems >= 4 * 2 * cap;
              if (!good) {
                std::printf("shape mismatch n=%d variant=%d cap=%d csize=%d lv=%d block=%d smem=%zu x=%d in=%d\n",
                            n, variant, cap, csize, lv, ls.block, ls.smem, ls.x_elems, ls.x_in_smem);
                return 1;
              }
            }
            ++cases;
          }
  // the circuit exporter's carve: flags (16-byte aligned), next times, counts
  for (int L : {1, 7, 16, 33, 4096}) {
    const size_t smem = static_cast<size_t>((L + 15) / 16) * 16 + static_cast<size_t>(L) * 12;
    const size_t tn = static_cast<size_t>((L + 15) / 16) * 16;
    if (tn % 8 != 0 || tn + static_cast<size_t>(L) * 8 + static_cast<size_t>(L) * 4 > smem || smem > kOptin) {
      std::printf("export carve mismatch L=%d\n", L);
      return 1;
    }
    ++cases;
  }
  std::printf("ok %ld\n", cases);
  return 0;
}
