// C ABI of the MTP library: handles, schedule upload and the entry points of include/mtp.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "mtp_internal.h"

namespace mtp {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

std::atomic<int> g_inject_alloc{0};
std::atomic<int> g_inject_overflow{0};
std::atomic<int> g_inject_grade_wait{0};

bool take_injected(std::atomic<int>& c) {
  int v = c.load();
  while (v > 0)
    if (c.compare_exchange_weak(v, v - 1)) return true;
  return false;
}

void DevBuf::ensure(size_t need, cudaStream_t s) {
  if (need == 0) need = 16;
  if (bytes >= need) return;
  if (take_injected(g_inject_alloc)) throw Fail{MTP_ERR_CUDA, "device allocation failed (injected fault)"};
  if (p) MTP_CUDA(cudaFreeAsync(p, s));
  p = nullptr;
  bytes = 0;
  size_t cap = need + need / 8;
  MTP_CUDA(cudaMallocAsync(&p, cap, s));
  bytes = cap;
}
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

namespace {

template <class T>
size_t put(std::vector<char>& blob, const std::vector<T>& v) {
  size_t off = (blob.size() + 255) & ~size_t(255);
  blob.resize(off + std::max<size_t>(v.size() * sizeof(T), 16));
  if (!v.empty()) std::memcpy(blob.data() + off, v.data(), v.size() * sizeof(T));
  return off;
}

}  // namespace

namespace {

// Orders the terms of one round (lists[l] for lanes l) into L iterations so that, at each
// iteration, the 32 lanes' two shared-memory operands fall into distinct banks as far as a
// greedy choice allows (same address = broadcast, free).  `bank_a/b` map a word to the
// word offset it reads; `swap` (optional) may exchange the two operands of a word.
template <class BankA, class BankB, class Swap>
std::vector<std::vector<uint32_t>> bank_order(std::vector<std::vector<uint32_t>> lists, int L, BankA bank_a,
                                              BankB bank_b, Swap swap) {
  std::vector<std::vector<uint32_t>> out(lists.size());
  for (int it = 0; it < L; ++it) {
    std::vector<std::vector<uint32_t>> addr_a(32), addr_b(32);
    auto cost = [&](uint32_t w) {
      const uint32_t oa = bank_a(w), ob = bank_b(w);
      int c = 0;
      auto& va = addr_a[oa & 31];
      if (std::find(va.begin(), va.end(), oa) == va.end()) c += static_cast<int>(va.size());
      auto& vb = addr_b[ob & 31];
      if (std::find(vb.begin(), vb.end(), ob) == vb.end()) c += static_cast<int>(vb.size());
      return c;
    };
    for (size_t l = 0; l < lists.size(); ++l) {
      auto& lst = lists[l];
      if (lst.empty()) continue;
      size_t best = 0;
      int bestc = 1 << 30;
      bool best_sw = false;
      for (size_t k = 0; k < lst.size(); ++k) {
        const int c0 = cost(lst[k]);
        if (c0 < bestc) { bestc = c0; best = k; best_sw = false; }
        const uint32_t ws = swap(lst[k]);
        if (ws != lst[k]) {
          const int c1 = cost(ws);
          if (c1 < bestc) { bestc = c1; best = k; best_sw = true; }
        }
        if (bestc == 0) break;
      }
      const uint32_t w = best_sw ? swap(lst[best]) : lst[best];
      lst.erase(lst.begin() + static_cast<long>(best));
      auto& va = addr_a[bank_a(w) & 31];
      if (std::find(va.begin(), va.end(), bank_a(w)) == va.end()) va.push_back(bank_a(w));
      auto& vb = addr_b[bank_b(w) & 31];
      if (std::find(vb.begin(), vb.end(), bank_b(w)) == vb.end()) vb.push_back(bank_b(w));
      out[l].push_back(w);
    }
  }
  return out;
}

}  // namespace

// Uploads the schedule with its forward waves (destinations grouped by dependency depth) and
// the transposed triple list for the adjoint (uses of each value, grouped by height).
void upload_schedule(mtp_model* md) {
  const Schedule& S = md->sched;
  const int nv = S.n_values, nm = S.n_mom_comps, nd = nv - nm;
  if (nv >= 65536) throw Fail{MTP_ERR_UNSUPPORTED, "value array exceeds 65535 entries"};
  std::vector<int> comp_info(nm);
  for (int c = 0; c < nm; ++c)
    comp_info[c] = S.comp_mu[c] | (S.comp_exp[c][0] << 8) | (S.comp_exp[c][1] << 16) | (S.comp_exp[c][2] << 24);
  std::vector<int> depth(nv, 0);
  for (int d = 0; d < nd; ++d) {
    int dep = 0;
    for (int t = S.dst_ptr[d]; t < S.dst_ptr[d + 1]; ++t)
      dep = std::max(dep, std::max(depth[S.tri_a[t]], depth[S.tri_b[t]]) + 1);
    depth[nm + d] = dep;
  }
  int maxdep = 0;
  for (int x = nm; x < nv; ++x) maxdep = std::max(maxdep, depth[x]);
  std::vector<int> fwave_ptr(1, 0), fdst;
  for (int w = 1; w <= maxdep; ++w) {
    std::vector<int> lst;
    for (int x = nm; x < nv; ++x)
      if (depth[x] == w) lst.push_back(x);
    std::stable_sort(lst.begin(), lst.end(), [&](int a, int b) {
      return (S.dst_ptr[a - nm + 1] - S.dst_ptr[a - nm]) > (S.dst_ptr[b - nm + 1] - S.dst_ptr[b - nm]);
    });
    fdst.insert(fdst.end(), lst.begin(), lst.end());
    fwave_ptr.push_back(static_cast<int>(fdst.size()));
  }
  std::vector<uint32_t> tri_ab(S.tri_a.size());
  std::vector<float> tri_cf(S.tri_a.size());
  for (size_t t = 0; t < S.tri_a.size(); ++t) {
    tri_ab[t] = static_cast<uint32_t>(S.tri_a[t]) | (static_cast<uint32_t>(S.tri_b[t]) << 16);
    tri_cf[t] = static_cast<float>(S.tri_c[t]);
  }
  // uses (gather form of the adjoint): d(c v_a v_b)/dv_a = c v_b, one entry per operand; a
  // square (a == b) gives the single entry 2 c v_a
  std::vector<std::vector<std::pair<uint32_t, double>>> uses(nv);
  for (int d = 0; d < nd; ++d)
    for (int t = S.dst_ptr[d]; t < S.dst_ptr[d + 1]; ++t) {
      const uint32_t dst = static_cast<uint32_t>(nm + d);
      if (S.tri_a[t] == S.tri_b[t]) {
        uses[S.tri_a[t]].push_back({static_cast<uint32_t>(S.tri_a[t]) | (dst << 16), 2.0 * S.tri_c[t]});
        continue;
      }
      uses[S.tri_a[t]].push_back({static_cast<uint32_t>(S.tri_b[t]) | (dst << 16), S.tri_c[t]});
      uses[S.tri_b[t]].push_back({static_cast<uint32_t>(S.tri_a[t]) | (dst << 16), S.tri_c[t]});
    }
  std::vector<int> height(nv, 0);
  for (int x = nv - 1; x >= 0; --x)
    for (auto& u : uses[x]) height[x] = std::max(height[x], height[u.first >> 16] + 1);
  int maxh = 0;
  for (int x = 0; x < nv; ++x) maxh = std::max(maxh, height[x]);
  std::vector<int> rwave_ptr(1, 0), rval;
  for (int h = 0; h <= maxh; ++h) {
    std::vector<int> lst;
    for (int x = 0; x < nv; ++x)
      if (height[x] == h) lst.push_back(x);
    std::stable_sort(lst.begin(), lst.end(), [&](int a, int b) { return uses[a].size() > uses[b].size(); });
    rval.insert(rval.end(), lst.begin(), lst.end());
    rwave_ptr.push_back(static_cast<int>(rval.size()));
  }
  std::vector<int> use_ptr(1, 0);
  std::vector<uint32_t> use_od;
  std::vector<double> use_cd;
  std::vector<float> use_cf;
  for (int x = 0; x < nv; ++x) {
    for (auto& u : uses[x]) { use_od.push_back(u.first); use_cd.push_back(u.second); use_cf.push_back(static_cast<float>(u.second)); }
    use_ptr.push_back(static_cast<int>(use_od.size()));
  }
  // packed words for the specialised kernel
  std::vector<double> coefs(S.tri_c.begin(), S.tri_c.end());
  coefs.insert(coefs.end(), use_cd.begin(), use_cd.end());
  std::sort(coefs.begin(), coefs.end());
  coefs.erase(std::unique(coefs.begin(), coefs.end()), coefs.end());
  const bool packable = nv <= 4096 && coefs.size() <= 255;
  std::vector<uint32_t> tri_pk, use_pk;
  std::vector<float> coef_f(coefs.begin(), coefs.end());
  coef_f.push_back(0.0f);   // coefficient of the padding terms
  const uint32_t zero_ci = static_cast<uint32_t>(coef_f.size() - 1);
  std::vector<uint32_t> fslab, rslab;
  std::vector<int> fr_dst, rr_val;
  std::vector<int> fround, rround;   // 4 ints per round
  // packed rounds for the three-kernel pass's contraction (same words): a long list may take an
  // aligned group of 2..32 lanes, each lane an equal share, combined by a butterfly; lane entry =
  // -1 (idle) or dst | log2(group) << 16 | leader << 20; round = {L, off, end_of_wave, grouped}
  std::vector<uint32_t> pfslab, prslab;
  std::vector<int> pfr_dst, prr_val, pfround, prround;
  if (packable) {
    auto ci = [&](double c) { return static_cast<uint32_t>(std::lower_bound(coefs.begin(), coefs.end(), c) - coefs.begin()); };
    for (size_t t = 0; t < S.tri_a.size(); ++t)
      tri_pk.push_back(static_cast<uint32_t>(S.tri_a[t]) | (static_cast<uint32_t>(S.tri_b[t]) << 12) | (ci(S.tri_c[t]) << 24));
    for (size_t u = 0; u < use_od.size(); ++u)
      use_pk.push_back((use_od[u] & 0xffffu) | ((use_od[u] >> 16) << 12) | (ci(use_cd[u]) << 24));
    const uint32_t pad = zero_ci << 24;   // 0 * v[0] * v[0]
    // forward slabs: waves of destinations, rounds of 32 (already sorted by length, descending)
    for (int wv = 0; wv + 1 < static_cast<int>(fwave_ptr.size()); ++wv)
      for (int e0 = fwave_ptr[wv]; e0 < fwave_ptr[wv + 1]; e0 += 32) {
        const int e1 = std::min(e0 + 32, fwave_ptr[wv + 1]);
        int L = 0;
        for (int e = e0; e < e1; ++e) L = std::max(L, S.dst_ptr[fdst[e] - nm + 1] - S.dst_ptr[fdst[e] - nm]);
        fround.insert(fround.end(), {L, static_cast<int>(fslab.size()), e1 == fwave_ptr[wv + 1] ? 1 : 0, 0});
        for (int l = 0; l < 32; ++l) fr_dst.push_back(e0 + l < e1 ? fdst[e0 + l] : -1);
        std::vector<std::vector<uint32_t>> lists(32);
        for (int e = e0; e < e1; ++e)
          for (int t = S.dst_ptr[fdst[e] - nm]; t < S.dst_ptr[fdst[e] - nm + 1]; ++t) lists[e - e0].push_back(tri_pk[t]);
        auto ord = bank_order(
            lists, L, [](uint32_t w) { return w & 4095u; }, [](uint32_t w) { return (w >> 12) & 4095u; },
            [](uint32_t w) { return (w & 0xff000000u) | ((w & 4095u) << 12) | ((w >> 12) & 4095u); });
        for (int it = 0; it < L; ++it)
          for (int l = 0; l < 32; ++l) fslab.push_back(it < static_cast<int>(ord[l].size()) ? ord[l][it] : pad);
      }
    // reverse slabs: waves of values by height, rounds of 32 (sorted by number of uses)
    for (int wv = 0; wv + 1 < static_cast<int>(rwave_ptr.size()); ++wv)
      for (int e0 = rwave_ptr[wv]; e0 < rwave_ptr[wv + 1]; e0 += 32) {
        const int e1 = std::min(e0 + 32, rwave_ptr[wv + 1]);
        int L = 0;
        for (int e = e0; e < e1; ++e) L = std::max(L, static_cast<int>(uses[rval[e]].size()));
        rround.insert(rround.end(), {L, static_cast<int>(rslab.size()), e1 == rwave_ptr[wv + 1] ? 1 : 0, 0});
        for (int l = 0; l < 32; ++l) rr_val.push_back(e0 + l < e1 ? rval[e0 + l] : -1);
        std::vector<std::vector<uint32_t>> lists(32);
        for (int e = e0; e < e1; ++e)
          for (int u = use_ptr[rval[e]]; u < use_ptr[rval[e] + 1]; ++u) lists[e - e0].push_back(use_pk[u]);
        const uint32_t gofs = static_cast<uint32_t>(padded_nv(nv));   // grads follow vals in shared memory
        auto ord = bank_order(
            lists, L, [](uint32_t w) { return w & 4095u; }, [gofs](uint32_t w) { return gofs + ((w >> 12) & 4095u); },
            [](uint32_t w) { return w; });
        for (int it = 0; it < L; ++it)
          for (int l = 0; l < 32; ++l) rslab.push_back(it < static_cast<int>(ord[l].size()) ? ord[l][it] : pad);
      }
    // packed rounds: items of one wave sorted by list length (descending); each round takes the
    // next items with group sizes g = next power of 2 of ceil(len / L) (aligned, non-increasing)
    // and the L that minimises (32 L + kRoundCost) per term, kRoundCost being the fixed cost of a
    // round in slot units
    auto pack_wave = [&](const std::vector<int>& items, auto&& list_of, std::vector<uint32_t>& slab,
                         std::vector<int>& lane_item, std::vector<int>& rounds, auto&& bank_a, auto&& bank_b,
                         auto&& swap) {
      constexpr double kRoundCost = 300.0;
      auto np2 = [](int x) { int g = 1; while (g < x) g *= 2; return g; };
      const int n = static_cast<int>(items.size());
      int i = 0;
      while (i < n) {
        const int len0 = static_cast<int>(list_of(items[i]).size());
        int bestL = -1, bestj = i + 1;
        double best_cost = 1e300;
        for (int g0 = 1; g0 <= 32; g0 *= 2) {
          const int L = len0 == 0 ? 0 : (len0 + g0 - 1) / g0;
          int lanes = 0, j = i;
          long long tot = 0;
          while (j < n) {
            const int len = static_cast<int>(list_of(items[j]).size());
            const int g = (L == 0 || len == 0) ? 1 : np2((len + L - 1) / L);
            if (L == 0 && len > 0) break;
            if (lanes + g > 32) break;
            lanes += g;
            tot += len;
            ++j;
          }
          if (j == i) continue;
          const double cost = L == 0 ? 0.0 : (32.0 * L + kRoundCost) / static_cast<double>(tot);
          if (bestL < 0 || cost < best_cost - 1e-12 || (std::abs(cost - best_cost) <= 1e-12 && j > bestj)) {
            best_cost = cost; bestL = L; bestj = j;
          }
        }
        const int L = bestL, j = bestj;
        std::vector<std::vector<uint32_t>> lists(32);
        std::vector<int> entry(32, -1);
        bool grouped = false;
        int lane = 0;
        for (int k = i; k < j; ++k) {
          const auto& lst = list_of(items[k]);
          const int len = static_cast<int>(lst.size());
          const int g = (L == 0 || len == 0) ? 1 : np2((len + L - 1) / L);
          int lg = 0;
          while ((1 << lg) < g) ++lg;
          if (g > 1) grouped = true;
          const int chunk = g > 1 ? (len + g - 1) / g : len;
          for (int q = 0; q < g; ++q) {
            for (int t = q * chunk; t < std::min(len, (q + 1) * chunk); ++t) lists[lane + q].push_back(lst[t]);
            entry[lane + q] = items[k] | (lg << 16) | ((q == 0 ? 1 : 0) << 20);
          }
          lane += g;
        }
        rounds.insert(rounds.end(), {L, static_cast<int>(slab.size()), j == n ? 1 : 0, grouped ? 1 : 0});
        lane_item.insert(lane_item.end(), entry.begin(), entry.end());
        auto ord = bank_order(lists, L, bank_a, bank_b, swap);
        for (int it = 0; it < L; ++it)
          for (int l = 0; l < 32; ++l) slab.push_back(it < static_cast<int>(ord[l].size()) ? ord[l][it] : pad);
        i = j;
      }
    };
    {
      std::vector<std::vector<uint32_t>> flist(nv);
      for (int x = nm; x < nv; ++x)
        for (int t = S.dst_ptr[x - nm]; t < S.dst_ptr[x - nm + 1]; ++t) flist[x].push_back(tri_pk[t]);
      std::vector<std::vector<uint32_t>> rlist(nv);
      for (int x = 0; x < nv; ++x)
        for (int u = use_ptr[x]; u < use_ptr[x + 1]; ++u) rlist[x].push_back(use_pk[u]);
      auto by_len = [&](std::vector<std::vector<uint32_t>>& L_, std::vector<int> items) {
        std::stable_sort(items.begin(), items.end(), [&](int a, int b) { return L_[a].size() > L_[b].size(); });
        return items;
      };
      const uint32_t gofs = static_cast<uint32_t>(padded_nv(nv));
      for (int wv = 0; wv + 1 < static_cast<int>(fwave_ptr.size()); ++wv) {
        std::vector<int> items(fdst.begin() + fwave_ptr[wv], fdst.begin() + fwave_ptr[wv + 1]);
        pack_wave(by_len(flist, items), [&](int x) -> const std::vector<uint32_t>& { return flist[x]; }, pfslab,
                  pfr_dst, pfround, [](uint32_t w) { return w & 4095u; }, [](uint32_t w) { return (w >> 12) & 4095u; },
                  [](uint32_t w) { return (w & 0xff000000u) | ((w & 4095u) << 12) | ((w >> 12) & 4095u); });
      }
      for (int wv = 0; wv + 1 < static_cast<int>(rwave_ptr.size()); ++wv) {
        std::vector<int> items(rval.begin() + rwave_ptr[wv], rval.begin() + rwave_ptr[wv + 1]);
        pack_wave(by_len(rlist, items), [&](int x) -> const std::vector<uint32_t>& { return rlist[x]; }, prslab,
                  prr_val, prround, [](uint32_t w) { return w & 4095u; },
                  [gofs](uint32_t w) { return gofs + ((w >> 12) & 4095u); }, [](uint32_t w) { return w; });
      }
    }
  }
  // inline coefficients when every coefficient is m 2^e with m < 128 (as the multinomial
  // weights of the contraction are) and the value indices fit 11 bits with the zero slot
  bool coef_inline = false;
  if (packable && nv + 1 <= 2048) {
    std::vector<uint32_t> code(coef_f.size(), 0u);
    bool ok = true;
    for (size_t k = 0; k + 1 < coef_f.size(); ++k) {
      const float c = coef_f[k];
      uint32_t bits;
      std::memcpy(&bits, &c, 4);
      const int e8 = static_cast<int>((bits >> 23) & 255u);
      if (!(c >= 1.0f) || static_cast<double>(c) != coefs[k] || (bits & 0x1FFFFu) != 0u || e8 > 127 + 15) {
        ok = false;
        break;
      }
      code[k] = (bits - 0x3F800000u) >> 17;   // 10 bits: exponent offset (4) and fraction (6)
    }
    if (ok) {
      const uint32_t z = static_cast<uint32_t>(nv);   // the always-zero value slot
      auto conv = [&](uint32_t w) {
        const uint32_t ci = w >> 24;
        if (ci == zero_ci) return z | (z << 11);     // 1 * 0 * 0
        return (w & 4095u) | (((w >> 12) & 4095u) << 11) | (code[ci] << 22);
      };
      for (auto& w : fslab) w = conv(w);
      for (auto& w : rslab) w = conv(w);
      for (auto& w : pfslab) w = conv(w);
      for (auto& w : prslab) w = conv(w);
      coef_inline = true;
    }
  }
  // every index the kernels will read from the schedule, checked on the host before upload
  {
    auto bad = [](const char* what) { throw Fail{MTP_ERR_NUMERIC, std::string("schedule index out of range: ") + what}; };
    const uint32_t ncf = static_cast<uint32_t>(coef_f.size());
    const uint32_t unv = static_cast<uint32_t>(nv);
    auto check_word = [&](uint32_t w, const char* what) {
      if (coef_inline) {
        if ((w & 2047u) > unv || ((w >> 11) & 2047u) > unv) bad(what);   // index nv = the zero slot
      } else if ((w & 4095u) >= unv || ((w >> 12) & 4095u) >= unv || (w >> 24) >= ncf) {
        bad(what);
      }
    };
    for (uint32_t w : fslab) check_word(w, "forward slab");
    for (uint32_t w : rslab) check_word(w, "reverse slab");
    for (uint32_t w : pfslab) check_word(w, "packed forward slab");
    for (uint32_t w : prslab) check_word(w, "packed reverse slab");
    auto check_packed = [&](const std::vector<int>& rounds, const std::vector<int>& entries, const std::vector<uint32_t>& slab,
                            int lo, const char* what) {
      if (entries.size() != 8 * rounds.size()) bad(what);
      for (size_t r = 0; r < rounds.size(); r += 4) {
        if (rounds[r] < 0 || rounds[r + 1] < 0 ||
            static_cast<size_t>(rounds[r + 1]) + 32 * static_cast<size_t>(rounds[r]) > slab.size())
          bad(what);
        for (int l = 0; l < 32; ++l) {
          const int e = entries[8 * r + l];
          if (e == -1) continue;
          const int x = e & 0xffff, lg = (e >> 16) & 15;
          if (x < lo || x >= nv || lg > 5 || (l & ((1 << lg) - 1)) != 0 && ((e >> 20) & 1)) bad(what);
        }
      }
    };
    check_packed(pfround, pfr_dst, pfslab, nm, "packed forward rounds");
    check_packed(prround, prr_val, prslab, 0, "packed reverse rounds");
    for (int x : fr_dst)
      if (x != -1 && (x < nm || x >= nv)) bad("forward destinations");
    for (int x : rr_val)
      if (x != -1 && (x < 0 || x >= nv)) bad("reverse values");
    for (size_t r = 0; r < fround.size(); r += 4)
      if (fround[r + 1] < 0 || static_cast<size_t>(fround[r + 1]) + 32 * static_cast<size_t>(fround[r]) > fslab.size())
        bad("forward rounds");
    for (size_t r = 0; r < rround.size(); r += 4)
      if (rround[r + 1] < 0 || static_cast<size_t>(rround[r + 1]) + 32 * static_cast<size_t>(rround[r]) > rslab.size())
        bad("reverse rounds");
    for (size_t t = 0; t < S.tri_a.size(); ++t)
      if (S.tri_a[t] < 0 || S.tri_a[t] >= nv || S.tri_b[t] < 0 || S.tri_b[t] >= nv) bad("triples");
    for (int x : S.basis_idx)
      if (x < 0 || x >= nv) bad("basis values");
  }
  std::vector<char> blob;
  const size_t o_tpk = put(blob, tri_pk), o_upk = put(blob, use_pk), o_cf = put(blob, coef_f);
  const size_t o_fs = put(blob, fslab), o_fr = put(blob, fround), o_frd = put(blob, fr_dst), o_rs = put(blob, rslab),
               o_rr = put(blob, rround), o_rrv = put(blob, rr_val);
  const size_t o_pfs = put(blob, pfslab), o_pfr = put(blob, pfround), o_pfd = put(blob, pfr_dst),
               o_prs = put(blob, prslab), o_prr = put(blob, prround), o_prv = put(blob, prr_val);
  const size_t o_ci = put(blob, comp_info), o_fwp = put(blob, fwave_ptr), o_fd = put(blob, fdst),
               o_tp = put(blob, S.dst_ptr), o_tab = put(blob, tri_ab), o_tcf = put(blob, tri_cf),
               o_tcd = put(blob, S.tri_c), o_rwp = put(blob, rwave_ptr), o_rv = put(blob, rval),
               o_up = put(blob, use_ptr), o_uod = put(blob, use_od), o_ucf = put(blob, use_cf),
               o_ucd = put(blob, use_cd), o_bi = put(blob, S.basis_idx);
  md->sched_buf.ensure(blob.size(), 0);
  MTP_CUDA(cudaMemcpy(md->sched_buf.p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  char* base = md->sched_buf.as<char>();
  DevSchedule& D = md->ds;
  D.n_types = S.n_types; D.n_q = S.n_q; D.n_rad = S.n_rad; D.n_lin = S.n_lin; D.n_params = S.n_params;
  D.n_mom = nm; D.n_vals = nv; D.first_dst = nm; D.nu_max = S.nu_max;
  D.n_fwaves = static_cast<int>(fwave_ptr.size()) - 1;
  D.n_rwaves = static_cast<int>(rwave_ptr.size()) - 1;
  D.r_min = md->desc.r_min; D.r_cut = md->desc.r_cut;
  D.comp_info = reinterpret_cast<const int*>(base + o_ci);
  D.fwave_ptr = reinterpret_cast<const int*>(base + o_fwp);
  D.fdst = reinterpret_cast<const int*>(base + o_fd);
  D.tri_ptr = reinterpret_cast<const int*>(base + o_tp);
  D.tri_ab = reinterpret_cast<const uint32_t*>(base + o_tab);
  D.tri_cf = reinterpret_cast<const float*>(base + o_tcf);
  D.tri_cd = reinterpret_cast<const double*>(base + o_tcd);
  D.rwave_ptr = reinterpret_cast<const int*>(base + o_rwp);
  D.rval = reinterpret_cast<const int*>(base + o_rv);
  D.use_ptr = reinterpret_cast<const int*>(base + o_up);
  D.use_od = reinterpret_cast<const uint32_t*>(base + o_uod);
  D.use_cf = reinterpret_cast<const float*>(base + o_ucf);
  D.use_cd = reinterpret_cast<const double*>(base + o_ucd);
  D.basis_idx = reinterpret_cast<const int*>(base + o_bi);
  D.tri_pk = packable ? reinterpret_cast<const uint32_t*>(base + o_tpk) : nullptr;
  D.use_pk = packable ? reinterpret_cast<const uint32_t*>(base + o_upk) : nullptr;
  D.coef_f = reinterpret_cast<const float*>(base + o_cf);
  D.coef_inline = coef_inline;
  D.n_coef = static_cast<int>(coef_f.size());
  D.n_tri = static_cast<int>(S.tri_a.size());
  D.fslab = reinterpret_cast<const uint32_t*>(base + o_fs);
  D.fround = reinterpret_cast<const int4*>(base + o_fr);
  D.fr_dst = reinterpret_cast<const int*>(base + o_frd);
  D.n_fround = static_cast<int>(fround.size() / 4);
  D.fslab_words = static_cast<int>(fslab.size());
  D.rslab = reinterpret_cast<const uint32_t*>(base + o_rs);
  D.rround = reinterpret_cast<const int4*>(base + o_rr);
  D.rr_val = reinterpret_cast<const int*>(base + o_rrv);
  D.n_rround = static_cast<int>(rround.size() / 4);
  D.rslab_words = static_cast<int>(rslab.size());
  D.n_use = static_cast<int>(use_od.size());
  D.pfslab = reinterpret_cast<const uint32_t*>(base + o_pfs);
  D.pfround = reinterpret_cast<const int4*>(base + o_pfr);
  D.pfr_dst = reinterpret_cast<const int*>(base + o_pfd);
  D.n_pfround = static_cast<int>(pfround.size() / 4);
  D.pfslab_words = static_cast<int>(pfslab.size());
  D.prslab = reinterpret_cast<const uint32_t*>(base + o_prs);
  D.prround = reinterpret_cast<const int4*>(base + o_prr);
  D.prr_val = reinterpret_cast<const int*>(base + o_prv);
  D.n_prround = static_cast<int>(prround.size() / 4);
  D.prslab_words = static_cast<int>(prslab.size());
}

void upload_theta(mtp_model* md) {
  const Schedule& S = md->sched;
  const int64_t m = S.n_params;
  std::vector<double> seed(S.n_values, 0.0);
  for (int a = 0; a < S.n_lin; ++a) seed[S.basis_idx[a]] += md->theta[S.n_types + a];
  std::vector<float> tf(m), sf(S.n_values);
  for (int64_t k = 0; k < m; ++k) tf[k] = static_cast<float>(md->theta[k]);
  for (int x = 0; x < S.n_values; ++x) sf[x] = static_cast<float>(seed[x]);
  std::vector<char> blob;
  const size_t o_td = put(blob, md->theta), o_tf = put(blob, tf), o_sd = put(blob, seed), o_sf = put(blob, sf);
  md->theta_buf.ensure(blob.size(), 0);
  MTP_CUDA(cudaMemcpy(md->theta_buf.p, blob.data(), blob.size(), cudaMemcpyHostToDevice));
  char* base = md->theta_buf.as<char>();
  md->ds.theta_d = reinterpret_cast<const double*>(base + o_td);
  md->ds.theta_f = reinterpret_cast<const float*>(base + o_tf);
  md->ds.seed_d = reinterpret_cast<const double*>(base + o_sd);
  md->ds.seed_f = reinterpret_cast<const float*>(base + o_sf);
}

void run_grade_simt(mtp_model* md, int64_t N, bool fp64, const double* rows, const float* rows_f, int64_t ld,
                    double* gamma, int32_t* argmax, cudaStream_t s);
bool grade_tc_available(const mtp_model* md);
void run_grade_tc(mtp_model* md, int64_t N, const float* hi, const float* lo, int64_t ld, double* gamma,
                  int32_t* argmax, const int32_t* zrow, const int64_t* row_atom, cudaStream_t s);

}  // namespace mtp

using namespace mtp;

namespace {

mtp_status fail(mtp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

template <class F>
mtp_status guarded(F&& f) {
  try {
    f();
    return MTP_OK;
  } catch (const Fail& e) {
    return fail(e.st, e.msg);
  } catch (const std::invalid_argument& e) {
    return fail(MTP_ERR_ARG, e.what());
  } catch (const std::bad_alloc&) {
    return fail(MTP_ERR_CUDA, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(MTP_ERR_CUDA, e.what());
  } catch (...) {
    return fail(MTP_ERR_CUDA, "unknown error");
  }
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

void check_desc(const mtp_desc* d) {
  if (!d) throw Fail{MTP_ERR_ARG, "null descriptor"};
  if (d->n_types < 1 || d->n_types > 64) throw Fail{MTP_ERR_ARG, "n_types must be in [1, 64]"};
  if (d->lev_max < 2 || d->lev_max > 28) throw Fail{MTP_ERR_ARG, "lev_max must be in [2, 28]"};
  if (d->n_q < 1 || d->n_q > 32) throw Fail{MTP_ERR_ARG, "n_q must be in [1, 32]"};
  if (!(d->r_cut > d->r_min) || !(d->r_min >= 0.0)) throw Fail{MTP_ERR_ARG, "need 0 <= r_min < r_cut"};
}

void fill_sizes(const Schedule& S, mtp_sizes* o) {
  o->n_params = S.n_params;
  o->n_lin = S.n_lin;
  o->n_rad = S.n_rad;
  o->n_moments = S.n_moments;
  o->n_mom_comps = S.n_mom_comps;
  o->n_values = S.n_values;
  o->n_triples = static_cast<int32_t>(S.tri_a.size());
  o->nu_max = S.nu_max;
  o->n_gauge = S.n_rad * (S.n_rad + 1) / 2;
}

void check_model(const mtp_model* m) {
  if (!m) throw Fail{MTP_ERR_ARG, "null model"};
  int dev = -1;
  MTP_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) throw Fail{MTP_ERR_ARG, "model belongs to another device"};
}

// Shared body of the EFS / grade / step entry points.
void efs_and_grade(mtp_model* m, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec, double* energy,
                   double* site_energy, double* forces, double* virial, double threshold, double* gamma,
                   int32_t* argmax, int32_t* flagged, int64_t* n_flagged, cudaStream_t s,
                   double* site_virial = nullptr) {
  check_run(m, b, nb);
  if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
  const bool fp64 = prec == MTP_FP64;
  const bool want_efs = energy || site_energy || forces || virial || site_virial;
  const bool want_grade = gamma != nullptr;
  if (!want_efs && !want_grade) throw Fail{MTP_ERR_ARG, "no output requested"};
  if ((flagged || n_flagged) && !gamma) throw Fail{MTP_ERR_ARG, "flagging needs gamma"};
  if (want_grade && !m->have_ainv) throw Fail{MTP_ERR_ARG, "no active set (call mtp_set_active_set)"};
  const int64_t N = nb->n_atoms, P = nb->n_pairs;
  SiteOutputs o;
  if (want_efs) {
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    m->ws_pair.ensure(std::max<int64_t>(P, 1) * 3 * rsz, s);
    m->ws_atom.ensure(N * 10 * sizeof(double), s);
    o.V = site_energy ? site_energy : m->ws_atom.as<double>();
    o.Wat = site_virial ? site_virial : m->ws_atom.as<double>() + N;
    o.G = m->ws_pair.p;
  }
  if (!fp64 && split_wanted(m)) {
    m->ws_mom.ensure(std::max<int64_t>(N, 1) * split_ldm(m->ds.n_mom) * sizeof(float), s);
    o.mom = m->ws_mom.as<float>();
  }
  int64_t ld = 0;
  const bool use_tc = !fp64 && want_grade && grade_tc_available(m);
  if (want_grade) {
    if (fp64) {
      ld = m->sched.n_params;
      m->ws_rows.ensure(N * ld * sizeof(double), s);
      o.rows = m->ws_rows.as<double>();
    } else if (use_tc) {
      ld = m->ainv_ld;
      m->ws_rows.ensure(2 * N * ld * sizeof(float), s);
      o.rows_hi = m->ws_rows.as<float>();
      o.rows_lo = o.rows_hi + N * ld;
    } else {
      ld = m->sched.n_params;
      m->ws_rows.ensure(N * ld * sizeof(float), s);
      o.rows_hi = m->ws_rows.as<float>();
    }
    o.rows_ld = ld;
  }
  // tensor-core grade with several species: the rows are stored in species order (the
  // neighborhoods are still evaluated in atom order), so that a row tile skips the radial blocks
  // of the species it does not hold; b_i and gamma_i are the same
  const int32_t* zrow = nullptr;
  const int64_t* row_atom = nullptr;
  if (use_tc && m->sched.n_types > 1) {
    m->ws_sort.ensure(N * (sizeof(int32_t) + 2 * sizeof(int64_t)) + 64, s);
    int64_t* order = m->ws_sort.as<int64_t>();
    int32_t* z = reinterpret_cast<int32_t*>(order + 2 * N);
    run_species_order(b->type, N, m->sched.n_types, z, order, m->ws_misc, s);
    o.row_pos = order + N;
    row_atom = order;
    zrow = z;
  }
  run_sites(m, b, nb, fp64, o, false, nullptr, s);
  if (want_efs) {
    if (forces) run_forces(nb, fp64, o.G, forces, s);
    if (energy || virial) run_config_sums(nb, o.V, o.Wat, energy, virial, m->ws_red, s);
  }
  if (want_grade) {
    if (use_tc) run_grade_tc(m, N, o.rows_hi, o.rows_lo, ld, gamma, argmax, zrow, row_atom, s);
    else run_grade_simt(m, N, fp64, o.rows, o.rows_hi, ld, gamma, argmax, s);
    if (flagged || n_flagged) {
      int64_t* cnt = n_flagged;
      int32_t* fl = flagged;
      if (!fl) {
        m->ws_misc.ensure(N * sizeof(int32_t) + 64, s);
        fl = m->ws_misc.as<int32_t>();
      }
      if (!cnt) throw Fail{MTP_ERR_ARG, "flagged needs n_flagged"};
      run_flag(N, gamma, threshold, fl, cnt, m->ws_red, s);
    }
  }
}

}  // namespace

namespace mtp {
void check_run(const mtp_model* m, const mtp_batch* b, const mtp_nbr* nb) {
  check_model(m);
  if (!b || !nb) throw Fail{MTP_ERR_ARG, "null batch or neighbor list"};
  if (b->n_cfg != nb->n_cfg) throw Fail{MTP_ERR_ARG, "neighbor list was built for another batch"};
  if (!b->pos || !b->type || !b->cell) throw Fail{MTP_ERR_ARG, "batch: null array"};
}
}  // namespace mtp

extern "C" {

const char* mtp_version(void) { return "mtp-gb300 1.0 (sm_103a)"; }
const char* mtp_last_error(void) { return g_last_error.c_str(); }

mtp_status mtp_describe(const mtp_desc* desc, mtp_sizes* out) {
  return guarded([&] {
    check_desc(desc);
    if (!out) throw Fail{MTP_ERR_ARG, "null output"};
    Schedule S = build_schedule(desc->n_types, desc->lev_max, desc->n_q);
    fill_sizes(S, out);
  });
}

mtp_status mtp_describe_basis(const mtp_desc* desc, int32_t* P, int32_t* mu, int32_t* nu, int32_t* edges) {
  return guarded([&] {
    check_desc(desc);
    if (!P || !mu || !nu || !edges) throw Fail{MTP_ERR_ARG, "null output"};
    Schedule S = build_schedule(desc->n_types, desc->lev_max, desc->n_q);
    for (int a = 0; a < S.n_lin; ++a) {
      P[a] = S.basis_P[a];
      for (int p = 0; p < 4; ++p) { mu[4 * a + p] = S.basis_mu[a][p]; nu[4 * a + p] = S.basis_nu[a][p]; }
      for (int e = 0; e < 6; ++e) edges[6 * a + e] = S.basis_edges[a][e];
    }
  });
}

mtp_status mtp_describe_schedule(const mtp_desc* desc, int32_t* comp_mu, int32_t* comp_exp, int32_t* dst_ptr,
                                 int32_t* tri_a, int32_t* tri_b, double* tri_c, int32_t* basis_idx) {
  return guarded([&] {
    check_desc(desc);
    Schedule S = build_schedule(desc->n_types, desc->lev_max, desc->n_q);
    if (comp_mu) for (int c = 0; c < S.n_mom_comps; ++c) comp_mu[c] = S.comp_mu[c];
    if (comp_exp)
      for (int c = 0; c < S.n_mom_comps; ++c)
        for (int q = 0; q < 3; ++q) comp_exp[3 * c + q] = S.comp_exp[c][q];
    if (dst_ptr) for (size_t k = 0; k < S.dst_ptr.size(); ++k) dst_ptr[k] = S.dst_ptr[k];
    if (tri_a) for (size_t t = 0; t < S.tri_a.size(); ++t) tri_a[t] = S.tri_a[t];
    if (tri_b) for (size_t t = 0; t < S.tri_b.size(); ++t) tri_b[t] = S.tri_b[t];
    if (tri_c) for (size_t t = 0; t < S.tri_c.size(); ++t) tri_c[t] = S.tri_c[t];
    if (basis_idx) for (int a = 0; a < S.n_lin; ++a) basis_idx[a] = S.basis_idx[a];
  });
}

mtp_status mtp_gauge_directions(const mtp_desc* desc, const double* theta, int64_t m, double* D) {
  return guarded([&] {
    check_desc(desc);
    if (!theta || !D) throw Fail{MTP_ERR_ARG, "null argument"};
    Schedule S = build_schedule(desc->n_types, desc->lev_max, desc->n_q);
    if (m != S.n_params) throw Fail{MTP_ERR_ARG, "theta size mismatch"};
    gauge_directions(S, theta, D);
  });
}

mtp_status mtp_load(const mtp_desc* desc, const double* theta, int64_t m, mtp_model** out) {
  return guarded([&] {
    check_desc(desc);
    if (!theta || !out) throw Fail{MTP_ERR_ARG, "null theta or output"};
    *out = nullptr;
    Schedule S = build_schedule(desc->n_types, desc->lev_max, desc->n_q);
    if (m != S.n_params)
      throw Fail{MTP_ERR_ARG, "theta has " + std::to_string(m) + " entries, the model needs " + std::to_string(S.n_params)};
    for (int64_t k = 0; k < m; ++k)
      if (!std::isfinite(theta[k])) throw Fail{MTP_ERR_NUMERIC, "non-finite theta"};
    auto* md = new mtp_model();
    try {
      MTP_CUDA(cudaGetDevice(&md->device));
      md->desc = *desc;
      md->sched = std::move(S);
      md->theta.assign(theta, theta + m);
      upload_schedule(md);
      upload_theta(md);
      split_prepare(md);
      noalloc_prepare(md->device);
      md->async_err.ensure(sizeof(unsigned), 0);
      MTP_CUDA(cudaMemset(md->async_err.p, 0, sizeof(unsigned)));
      MTP_CUDA(cudaDeviceSynchronize());
    } catch (...) {
      mtp_free_model(md);
      throw;
    }
    *out = md;
  });
}

void mtp_free_model(mtp_model* md) {
  if (!md) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(md->device);
  cudaDeviceSynchronize();
  for (DevBuf* b : {&md->sched_buf, &md->theta_buf, &md->a_d, &md->ainv_d, &md->ainv_f, &md->ws_pair,
                    &md->ws_atom, &md->ws_rows, &md->ws_grade, &md->ws_sort, &md->ws_misc, &md->ws_red,
                    &md->err_flag, &md->async_err, &md->split_tab, &md->ws_mom})
    b->release();
  cudaSetDevice(cur);
  delete md;
}

int64_t mtp_num_params(const mtp_model* md) { return md ? md->sched.n_params : -1; }

mtp_status mtp_model_sizes(const mtp_model* md, mtp_sizes* out) {
  return guarded([&] {
    if (!md || !out) throw Fail{MTP_ERR_ARG, "null argument"};
    fill_sizes(md->sched, out);
  });
}

mtp_status mtp_set_params(mtp_model* md, const double* theta, int64_t m) {
  return guarded([&] {
    check_model(md);
    if (!theta || m != md->sched.n_params) throw Fail{MTP_ERR_ARG, "theta size mismatch"};
    for (int64_t k = 0; k < m; ++k)
      if (!std::isfinite(theta[k])) throw Fail{MTP_ERR_NUMERIC, "non-finite theta"};
    MTP_CUDA(cudaDeviceSynchronize());
    md->theta.assign(theta, theta + m);
    upload_theta(md);
  });
}

mtp_status mtp_autotune(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec, int32_t* warps,
                        double* ms, void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
    cudaStream_t s = as_stream(stream);
    const int64_t N = nb->n_atoms, K = nb->n_cfg;
    DevBuf out;
    out.ensure((K * 10 + 4 * std::max<int64_t>(N, 1)) * sizeof(double) + 64, s);
    double* E = out.as<double>();
    double* W = E + K;
    double* F = W + 9 * K;
    double* gam = F + 3 * std::max<int64_t>(N, 1);
    double* gamma = md->have_ainv ? gam : nullptr;
    // the pass that mtp_step makes (energies, forces, virial and, with an active set, the grade)
    auto run = [&] { efs_and_grade(md, b, nb, prec, E, nullptr, F, W, 0.0, gamma, nullptr, nullptr, nullptr, s); };
    // the first pass (default shape) shows which kernel this precision runs; the other kernel's
    // tuned shape is kept
    const int keep_fast = md->tune_warps_fast, keep_fwd = md->tune_fwd_global, keep_gen = md->tune_warps_generic;
    md->tune_warps_fast = md->tune_warps_generic = 0;
    md->tune_fwd_global = -1;
    run();
    const bool fast = md->last_fast;
    if (fast) {
      md->tune_warps_generic = keep_gen;
    } else {
      md->tune_warps_fast = keep_fast;
      md->tune_fwd_global = keep_fwd;
    }
    int& knob = fast ? md->tune_warps_fast : md->tune_warps_generic;
    const int max_w = fast ? 8 : 4;
    // the three-kernel pass replaces the generic kernel in mixed precision where the shape has
    // one: the generic kernel is then timed at its default shape only (seconds per pass at
    // level 24)
    const bool split_ok = md->split_tab.p && prec == MTP_MIXED && md->mixed_pass != 1;
    const int min_w = (!fast && split_ok) ? max_w : 1;
    cudaEvent_t e0, e1;
    MTP_CUDA(cudaEventCreate(&e0));
    MTP_CUDA(cudaEventCreate(&e1));
    int best_w = 0, best_p = -1;
    float best_ms = 0.f;
    const int keep_pass = md->mixed_pass;
    if (fast && keep_pass != 2) md->mixed_pass = 1;   // the single-kernel shapes first
    struct Restore { mtp_model* m; int v; ~Restore() { m->mixed_pass = v; } } restore{md, keep_pass};
    // candidate shapes: (forward-slab placement, warps per block); the generic kernel has only warps
    for (int place = 0; place < (fast ? 2 : 1); ++place) {
      if (fast) md->tune_fwd_global = place;
      int last_used = -1;
      for (int w = max_w; w >= min_w; --w) {
        knob = w;
        run();   // warm-up at this shape
        if (fast && static_cast<int>(md->last_fwd_global) != place) break;   // placement unavailable
        if (md->last_warps == last_used) continue;   // clamped to a shape already timed
        last_used = md->last_warps;
        float t_min = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
          MTP_CUDA(cudaEventRecord(e0, s));
          run();
          MTP_CUDA(cudaEventRecord(e1, s));
          MTP_CUDA(cudaEventSynchronize(e1));
          float t = 0.f;
          MTP_CUDA(cudaEventElapsedTime(&t, e0, e1));
          if (rep == 0 || t < t_min) t_min = t;
        }
        if (best_w == 0 || t_min < best_ms) { best_ms = t_min; best_w = md->last_warps; best_p = place; }
      }
    }
    // the three-kernel mixed pass, when the model has one: warps per block of its per-pair
    // kernels x neighborhoods per warp of its contraction x words in flight x schedule placement
    // (results are the same for every shape)
    int best_sw = 0, best_snb = 0, best_sun = 0, best_sg = 0;
    float best_split = 0.f;
    const int keep_split = md->tune_split;
    md->mixed_pass = keep_pass;
    if (split_ok) {
      md->tune_split = 1;
      for (int sg : {1, 2, 3})
      for (int sw : {4, 8})
        for (int sc : {12, 14, 22, 24, 28}) {
          const int snb = sc / 10, sun = sc % 10;
          // level 24 (6 radial functions): only the streamed schedule applies
          if (md->ds.n_rad >= 6 && (sg != 2 || sun == 8)) continue;
          md->tune_split_warps = sw;
          md->tune_split_nb = snb;
          md->tune_split_unroll = sun;
          md->tune_split_sched = sg;
          run();
          if (!md->last_split || md->last_split_sched != sg) continue;   // placement unavailable
          float t_min = 0.f;
          for (int rep = 0; rep < 3; ++rep) {
            MTP_CUDA(cudaEventRecord(e0, s));
            run();
            MTP_CUDA(cudaEventRecord(e1, s));
            MTP_CUDA(cudaEventSynchronize(e1));
            float t = 0.f;
            MTP_CUDA(cudaEventElapsedTime(&t, e0, e1));
            if (rep == 0 || t < t_min) t_min = t;
          }
          if (best_sw == 0 || t_min < best_split) {
            best_split = t_min; best_sw = sw; best_snb = snb; best_sun = sun; best_sg = sg;
          }
        }
      md->tune_split = keep_split;
    }
    MTP_CUDA(cudaEventDestroy(e0));
    MTP_CUDA(cudaEventDestroy(e1));
    knob = best_w;
    if (fast) md->tune_fwd_global = best_p;
    if (best_sw > 0) {
      md->tune_split_warps = best_sw;
      md->tune_split_nb = best_snb;
      md->tune_split_unroll = best_sun;
      md->tune_split_sched = best_sg;
      const bool split = md->mixed_pass == 2 || best_split < best_ms;
      if (md->mixed_pass == 0) md->tune_split = split ? 1 : 0;
      if (split) best_ms = best_split;
    }
    MTP_CUDA(cudaStreamSynchronize(s));
    if (warps) *warps = best_w;
    if (ms) *ms = best_ms;
  });
}

mtp_status mtp_get_launch_shape(const mtp_model* md, int32_t* warps_fast, int32_t* fwd_global,
                                int32_t* warps_generic) {
  return guarded([&] {
    if (!md) throw Fail{MTP_ERR_ARG, "null model"};
    if (warps_fast) *warps_fast = md->tune_warps_fast;
    if (fwd_global) *fwd_global = md->tune_fwd_global;
    if (warps_generic) *warps_generic = md->tune_warps_generic;
  });
}

mtp_status mtp_set_mixed_pass(mtp_model* md, int pass) {
  return guarded([&] {
    check_model(md);
    if (pass < 0 || pass > 2) throw Fail{MTP_ERR_ARG, "pass must be 0 (automatic), 1 (single kernel) or 2 (three kernels)"};
    if (pass == 2 && !md->split_tab.p) throw Fail{MTP_ERR_UNSUPPORTED, "no three-kernel pass for this model's shape"};
    md->mixed_pass = pass;
  });
}

mtp_status mtp_set_split_shape(mtp_model* md, int warps_pair, int nb_contract, int unroll, int schedule) {
  return guarded([&] {
    check_model(md);
    if (warps_pair != 0 && warps_pair != 4 && warps_pair != 8) throw Fail{MTP_ERR_ARG, "warps_pair must be 0, 4 or 8"};
    if (nb_contract < 0 || nb_contract > 2) throw Fail{MTP_ERR_ARG, "nb_contract must be 0, 1 or 2"};
    if (unroll != 0 && unroll != 2 && unroll != 4 && unroll != 8) throw Fail{MTP_ERR_ARG, "unroll must be 0, 2, 4 or 8"};
    if (schedule < 0 || schedule > 3) throw Fail{MTP_ERR_ARG, "schedule must be 0, 1, 2 or 3"};
    md->tune_split_warps = warps_pair;
    md->tune_split_nb = nb_contract;
    md->tune_split_unroll = unroll;
    md->tune_split_sched = schedule;
  });
}

mtp_status mtp_get_split_shape(const mtp_model* md, int32_t* warps_pair, int32_t* nb_contract, int32_t* unroll,
                               int32_t* schedule, int32_t* schedule_used) {
  return guarded([&] {
    if (!md) throw Fail{MTP_ERR_ARG, "null model"};
    if (warps_pair) *warps_pair = md->tune_split_warps;
    if (nb_contract) *nb_contract = md->tune_split_nb;
    if (unroll) *unroll = md->tune_split_unroll;
    if (schedule) *schedule = md->tune_split_sched;
    if (schedule_used) *schedule_used = md->last_split_sched;
  });
}

mtp_status mtp_get_mixed_pass(const mtp_model* md, int32_t* setting, int32_t* in_use, int32_t* split_warps,
                              int32_t* split_nb) {
  return guarded([&] {
    if (!md) throw Fail{MTP_ERR_ARG, "null model"};
    if (setting) *setting = md->mixed_pass;
    if (in_use) *in_use = split_wanted(md) ? 2 : 1;
    if (split_warps) *split_warps = md->tune_split_warps;
    if (split_nb) *split_nb = md->tune_split_nb;
  });
}

mtp_status mtp_get_params(const mtp_model* md, double* theta, int64_t m) {
  return guarded([&] {
    check_model(md);
    if (!theta || m != md->sched.n_params) throw Fail{MTP_ERR_ARG, "theta size mismatch"};
    std::copy(md->theta.begin(), md->theta.end(), theta);
  });
}

namespace {
constexpr uint32_t kBlobMagic = 0x3150544du;   // "MTP1"
constexpr uint32_t kBlobVersion = 1u;
}  // namespace

mtp_status mtp_save(const mtp_model* md, void* buffer, int64_t capacity, int64_t* size, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!size) throw Fail{MTP_ERR_ARG, "null size"};
    const int64_t m = md->sched.n_params;
    const bool with_a = md->have_ainv;
    const int64_t need = 8 + static_cast<int64_t>(sizeof(mtp_desc)) + 8 + 8 * m + 8 + (with_a ? 8 * m * m : 0);
    *size = need;
    if (!buffer) return;
    if (capacity < need) throw Fail{MTP_ERR_CAPACITY, "checkpoint needs " + std::to_string(need) + " bytes"};
    unsigned char* p = static_cast<unsigned char*>(buffer);
    auto put_bytes = [&](const void* src, size_t n) { std::memcpy(p, src, n); p += n; };
    const uint32_t head[2] = {kBlobMagic, kBlobVersion};
    put_bytes(head, 8);
    put_bytes(&md->desc, sizeof(mtp_desc));
    put_bytes(&m, 8);
    put_bytes(md->theta.data(), 8 * m);
    const int64_t flag = with_a ? 1 : 0;
    put_bytes(&flag, 8);
    if (with_a) {
      MTP_CUDA(cudaMemcpyAsync(p, md->a_d.p, 8 * m * m, cudaMemcpyDeviceToHost, as_stream(stream)));
      MTP_CUDA(cudaStreamSynchronize(as_stream(stream)));
    }
  });
}

mtp_status mtp_restore(const void* buffer, int64_t size, mtp_model** out, void* stream) {
  mtp_model* md = nullptr;
  const mtp_status st = guarded([&] {
    if (!buffer || !out) throw Fail{MTP_ERR_ARG, "null argument"};
    if (size < 0) throw Fail{MTP_ERR_ARG, "negative size"};
    const unsigned char* p = static_cast<const unsigned char*>(buffer);
    const unsigned char* end = p + size;
    auto get = [&](void* dst, size_t n) {
      if (static_cast<size_t>(end - p) < n) throw Fail{MTP_ERR_ARG, "truncated checkpoint"};
      std::memcpy(dst, p, n);
      p += n;
    };
    uint32_t head[2];
    get(head, 8);
    if (head[0] != kBlobMagic || head[1] != kBlobVersion) throw Fail{MTP_ERR_ARG, "not an MTP checkpoint"};
    mtp_desc d;
    get(&d, sizeof(mtp_desc));
    int64_t m = 0;
    get(&m, 8);
    if (m <= 0 || m > (1 << 20)) throw Fail{MTP_ERR_ARG, "bad parameter count"};
    std::vector<double> theta(static_cast<size_t>(m));
    get(theta.data(), 8 * m);
    int64_t flag = 0;
    get(&flag, 8);
    std::vector<double> A;
    if (flag) {
      A.resize(static_cast<size_t>(m * m));
      get(A.data(), 8 * m * m);
    }
    const mtp_status s1 = mtp_load(&d, theta.data(), m, &md);
    if (s1 != MTP_OK) throw Fail{s1, mtp_last_error()};
    if (flag) {
      cudaStream_t s = as_stream(stream);
      DevBuf dA;
      dA.ensure(8 * m * m, s);
      MTP_CUDA(cudaMemcpyAsync(dA.p, A.data(), 8 * m * m, cudaMemcpyHostToDevice, s));
      const mtp_status s2 = mtp_set_active_set(md, dA.as<double>(), m, stream);
      MTP_CUDA(cudaStreamSynchronize(s));
      dA.release();
      if (s2 != MTP_OK) throw Fail{s2, mtp_last_error()};
    }
    *out = md;
  });
  if (st != MTP_OK && md) mtp_free_model(md);
  return st;
}

mtp_status mtp_debug_inject(int fault, int count) {
  return guarded([&] {
    if (count < 0) throw Fail{MTP_ERR_ARG, "negative count"};
    if (fault == MTP_FAULT_DEVICE_ALLOC) g_inject_alloc = count;
    else if (fault == MTP_FAULT_NEIGHBOR_OVERFLOW) g_inject_overflow = count;
    else if (fault == MTP_FAULT_GRADE_WAIT) g_inject_grade_wait = count;
    else throw Fail{MTP_ERR_ARG, "unknown fault"};
  });
}

mtp_status mtp_sync(mtp_model* md, void* stream) {
  return guarded([&] {
    check_model(md);
    cudaStream_t s = as_stream(stream);
    unsigned flag = 0;
    MTP_CUDA(cudaMemcpyAsync(&flag, md->async_err.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    MTP_CUDA(cudaStreamSynchronize(s));
    if (flag) {
      MTP_CUDA(cudaMemsetAsync(md->async_err.p, 0, sizeof(unsigned), s));
      MTP_CUDA(cudaStreamSynchronize(s));
      throw Fail{MTP_ERR_TIMEOUT, "a bounded wait of the tensor-core grade expired; the grades it did not finish are NaN"};
    }
  });
}

mtp_status mtp_set_active_set(mtp_model* md, const double* A, int64_t m, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!A || m != md->sched.n_params) throw Fail{MTP_ERR_ARG, "active-set matrix must be m x m"};
    md->have_ainv = false;
    cudaStream_t s = as_stream(stream);
    md->a_d.ensure(m * m * sizeof(double), s);
    MTP_CUDA(cudaMemcpyAsync(md->a_d.p, A, m * m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    run_lu_inverse(md, md->a_d.as<double>(), m, s);
  });
}

mtp_status mtp_get_active_set(const mtp_model* md, double* A, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!md->have_ainv || !A) throw Fail{MTP_ERR_ARG, "no active set or null output"};
    MTP_CUDA(cudaMemcpyAsync(A, md->a_d.p, md->m_active * md->m_active * sizeof(double), cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
  });
}

mtp_status mtp_maxvol(mtp_model* md, const double* B, int64_t n, double eps, int64_t max_swaps, int64_t* source,
                      int64_t* n_swaps, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!md->have_ainv) throw Fail{MTP_ERR_ARG, "no active set (call mtp_set_active_set)"};
    if (n < 0 || (n > 0 && !B)) throw Fail{MTP_ERR_ARG, "null or negative candidate rows"};
    if (!(eps >= 0.0) || max_swaps < 0) throw Fail{MTP_ERR_ARG, "eps and max_swaps must be non-negative"};
    const int64_t k = run_maxvol(md, B, n, eps, max_swaps, source, as_stream(stream));
    if (n_swaps) *n_swaps = k;
  });
}

mtp_status mtp_get_active_inverse(const mtp_model* md, double* Ainv, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!md->have_ainv || !Ainv) throw Fail{MTP_ERR_ARG, "no active set or null output"};
    MTP_CUDA(cudaMemcpyAsync(Ainv, md->ainv_d.p, md->m_active * md->m_active * sizeof(double),
                             cudaMemcpyDeviceToDevice, as_stream(stream)));
  });
}

mtp_status mtp_build_neighbors(mtp_model* md, const mtp_batch* b, mtp_nbr** inout, void* stream) {
  return guarded([&] {
    check_model(md);
    if (!inout) throw Fail{MTP_ERR_ARG, "null neighbor-list pointer"};
    mtp_nbr* nb = *inout;
    bool fresh = false;
    if (!nb) { nb = new mtp_nbr(); fresh = true; MTP_CUDA(cudaGetDevice(&nb->device)); }
    try {
      build_neighbors(md, b, nb, as_stream(stream));
    } catch (...) {
      if (fresh) mtp_free_nbr(nb);
      throw;
    }
    *inout = nb;
  });
}

void mtp_free_nbr(mtp_nbr* nb) {
  if (!nb) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(nb->device);
  cudaDeviceSynchronize();
  for (DevBuf* b : {&nb->off, &nb->pj, &nb->pimg, &nb->prev, &nb->pr32, &nb->atom_cfg, &nb->segs, &nb->masks,
                    &nb->bins, &nb->plan, &nb->shifts, &nb->wrap, &nb->scratch, &nb->counts, &nb->seg})
    b->release();
  cudaSetDevice(cur);
  delete nb;
}

mtp_status mtp_nbr_size(const mtp_nbr* nb, int64_t* n_atoms, int64_t* n_pairs) {
  return guarded([&] {
    if (!nb) throw Fail{MTP_ERR_ARG, "null neighbor list"};
    if (n_atoms) *n_atoms = nb->n_atoms;
    if (n_pairs) *n_pairs = nb->n_pairs;
  });
}

mtp_status mtp_nbr_reverse(const mtp_nbr* nb, int32_t* rev, void* stream) {
  return guarded([&] {
    if (!nb) throw Fail{MTP_ERR_ARG, "null neighbor list"};
    if (nb->n_pairs == 0) return;
    if (!rev) throw Fail{MTP_ERR_ARG, "null rev"};
    MTP_CUDA(cudaMemcpyAsync(rev, nb->prev.p, nb->n_pairs * sizeof(int32_t), cudaMemcpyDeviceToDevice, as_stream(stream)));
  });
}

mtp_status mtp_nbr_export(const mtp_nbr* nb, const mtp_batch* b, int64_t* off, int32_t* j, int32_t* image, double* r,
                          void* stream) {
  return guarded([&] {
    if (!nb) throw Fail{MTP_ERR_ARG, "null neighbor list"};
    cudaStream_t s = as_stream(stream);
    if (off) MTP_CUDA(cudaMemcpyAsync(off, nb->off.p, (nb->n_atoms + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    if (j && nb->n_pairs) MTP_CUDA(cudaMemcpyAsync(j, nb->pj.p, nb->n_pairs * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    if (image || r) {
      // unpack via the extraction kernel over all atoms would need an index list; do it on the host side
      std::vector<int> pimg(nb->n_pairs), pj(nb->n_pairs), cfg(nb->n_atoms);
      std::vector<long long> o(nb->n_atoms + 1);
      MTP_CUDA(cudaMemcpyAsync(pimg.data(), nb->pimg.p, nb->n_pairs * sizeof(int), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaMemcpyAsync(pj.data(), nb->pj.p, nb->n_pairs * sizeof(int), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaMemcpyAsync(cfg.data(), nb->atom_cfg.p, nb->n_atoms * sizeof(int), cudaMemcpyDeviceToHost, s));
      MTP_CUDA(cudaMemcpyAsync(o.data(), nb->off.p, o.size() * sizeof(long long), cudaMemcpyDeviceToHost, s));
      std::vector<double> pos, cell;
      if (r) {
        if (!b) throw Fail{MTP_ERR_ARG, "exporting r needs the batch"};
        pos.resize(3 * nb->n_atoms);
        cell.resize(9 * nb->n_cfg);
        MTP_CUDA(cudaMemcpyAsync(pos.data(), b->pos, pos.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        MTP_CUDA(cudaMemcpyAsync(cell.data(), b->cell, cell.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
      }
      MTP_CUDA(cudaStreamSynchronize(s));
      std::vector<int> img3(3 * nb->n_pairs);
      std::vector<double> r3(r ? 3 * nb->n_pairs : 0);
      for (int64_t i = 0; i < nb->n_atoms; ++i)
        for (long long p = o[i]; p < o[i + 1]; ++p) {
          const int n0 = unpack_img(pimg[p], 0), n1 = unpack_img(pimg[p], 1), n2 = unpack_img(pimg[p], 2);
          img3[3 * p] = n0; img3[3 * p + 1] = n1; img3[3 * p + 2] = n2;
          if (r) {
            const double* H = &cell[9 * cfg[i]];
            for (int c = 0; c < 3; ++c) {
              const double sh = n0 * H[c] + n1 * H[3 + c] + n2 * H[6 + c];
              r3[3 * p + c] = (pos[3 * pj[p] + c] + sh) - pos[3 * i + c];
            }
          }
        }
      if (image) MTP_CUDA(cudaMemcpyAsync(image, img3.data(), img3.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      if (r) MTP_CUDA(cudaMemcpyAsync(r, r3.data(), r3.size() * sizeof(double), cudaMemcpyHostToDevice, s));
      MTP_CUDA(cudaStreamSynchronize(s));
    }
  });
}

mtp_status mtp_energy_forces_stress(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                                    double* energy, double* site_energy, double* forces, double* virial,
                                    void* stream) {
  return guarded([&] {
    efs_and_grade(md, b, nb, prec, energy, site_energy, forces, virial, 0.0, nullptr, nullptr, nullptr, nullptr,
                  as_stream(stream));
  });
}

mtp_status mtp_energy_forces_stress_atoms(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                                          double* energy, double* site_energy, double* forces, double* virial,
                                          double* site_virial, void* stream) {
  return guarded([&] {
    efs_and_grade(md, b, nb, prec, energy, site_energy, forces, virial, 0.0, nullptr, nullptr, nullptr, nullptr,
                  as_stream(stream), site_virial);
  });
}

mtp_status mtp_grade(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec, double threshold,
                     double* gamma, int32_t* argmax, int32_t* flagged, int64_t* n_flagged, void* stream) {
  return guarded([&] {
    if (!gamma) throw Fail{MTP_ERR_ARG, "null gamma"};
    efs_and_grade(md, b, nb, prec, nullptr, nullptr, nullptr, nullptr, threshold, gamma, argmax, flagged, n_flagged,
                  as_stream(stream));
  });
}

mtp_status mtp_config_rows(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec, double* rows,
                           void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
    if (!rows) throw Fail{MTP_ERR_ARG, "null rows"};
    cudaStream_t s = as_stream(stream);
    const int64_t m = md->sched.n_params, N = nb->n_atoms;
    md->ws_rows.ensure(std::max<int64_t>(N, 1) * m * sizeof(double), s);
    SiteOutputs o;
    o.rows = md->ws_rows.as<double>();
    o.rows_ld = m;
    run_sites(md, b, nb, prec == MTP_FP64, o, false, nullptr, s);
    run_config_row_sums(nb, md->ws_rows.as<double>(), m, rows, md->ws_red, s);
  });
}

mtp_status mtp_energy_vjp(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                          const double* gE, const double* forces, double* g_pos, double* g_theta, void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
    if (!gE || (!g_pos && !g_theta)) throw Fail{MTP_ERR_ARG, "null gE or no output requested"};
    if (g_pos && !forces) throw Fail{MTP_ERR_ARG, "g_pos needs the forces of the forward pass"};
    cudaStream_t s = as_stream(stream);
    const int64_t m = md->sched.n_params, N = nb->n_atoms, K = nb->n_cfg;
    DevBuf work;
    double* R = nullptr;
    if (g_theta) {
      work.ensure(std::max<int64_t>(K, 1) * m * sizeof(double), s);
      R = work.as<double>();
      md->ws_rows.ensure(std::max<int64_t>(N, 1) * m * sizeof(double), s);
      SiteOutputs o;
      o.rows = md->ws_rows.as<double>();
      o.rows_ld = m;
      run_sites(md, b, nb, prec == MTP_FP64, o, false, nullptr, s);
      run_config_row_sums(nb, md->ws_rows.as<double>(), m, R, md->ws_red, s);
    }
    run_energy_vjp(nb, R, gE, m, forces, g_pos, g_theta, s);
    MTP_CUDA(cudaStreamSynchronize(s));   // `work` is released on return
  });
}

mtp_status mtp_config_grade(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                            mtp_grade_mode mode, double gamma_save, double gamma_break, double* gamma_cfg,
                            int64_t* worst, int32_t* cls, void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (!gamma_cfg) throw Fail{MTP_ERR_ARG, "null gamma_cfg"};
    if (mode != MTP_GRADE_NEIGHBORHOOD && mode != MTP_GRADE_CONFIGURATION) throw Fail{MTP_ERR_ARG, "unknown mode"};
    if (!md->have_ainv) throw Fail{MTP_ERR_ARG, "no active set (call mtp_set_active_set)"};
    cudaStream_t s = as_stream(stream);
    const int64_t m = md->sched.n_params, K = nb->n_cfg;
    DevBuf work;
    if (mode == MTP_GRADE_NEIGHBORHOOD) {
      work.ensure(std::max<int64_t>(nb->n_atoms, 1) * sizeof(double), s);
      efs_and_grade(md, b, nb, prec, nullptr, nullptr, nullptr, nullptr, 0.0, work.as<double>(), nullptr, nullptr,
                    nullptr, s);
      run_config_gamma_max(nb, work.as<double>(), gamma_cfg, worst, md->ws_misc, s);
    } else {
      if (prec != MTP_FP64 && prec != MTP_MIXED) throw Fail{MTP_ERR_ARG, "unknown precision"};
      work.ensure(std::max<int64_t>(K, 1) * (m * sizeof(double) + sizeof(int32_t)) + 64, s);
      double* rc = work.as<double>();
      int32_t* am = reinterpret_cast<int32_t*>(rc + std::max<int64_t>(K, 1) * m);
      const int64_t N = nb->n_atoms;
      md->ws_rows.ensure(std::max<int64_t>(N, 1) * m * sizeof(double), s);
      SiteOutputs o;
      o.rows = md->ws_rows.as<double>();
      o.rows_ld = m;
      run_sites(md, b, nb, prec == MTP_FP64, o, false, nullptr, s);
      run_config_row_sums(nb, md->ws_rows.as<double>(), m, rc, md->ws_red, s);
      run_grade_simt(md, K, true, rc, nullptr, m, gamma_cfg, am, s);
      if (worst) run_widen_argmax(am, K, worst, s);
    }
    if (cls) run_classify(gamma_cfg, K, gamma_save, gamma_break, cls, s);
    MTP_CUDA(cudaStreamSynchronize(s));
  });
}

mtp_status mtp_step(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec, double* energy,
                    double* site_energy, double* forces, double* virial, double threshold, double* gamma,
                    int32_t* argmax, int32_t* flagged, int64_t* n_flagged, void* stream) {
  return guarded([&] {
    efs_and_grade(md, b, nb, prec, energy, site_energy, forces, virial, threshold, gamma, argmax, flagged, n_flagged,
                  as_stream(stream));
  });
}

mtp_status mtp_param_rows(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                          const int64_t* atoms, int64_t n, double* rows, void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (!rows) throw Fail{MTP_ERR_ARG, "null rows"};
    if (atoms && n < 0) throw Fail{MTP_ERR_ARG, "negative count"};
    SiteOutputs o;
    o.rows = rows;
    o.rows_ld = md->sched.n_params;
    o.atom_list = atoms;
    o.n_list = atoms ? n : nb->n_atoms;
    run_sites(md, b, nb, prec == MTP_FP64, o, false, nullptr, as_stream(stream));
  });
}

mtp_status mtp_extract_neighborhoods(const mtp_nbr* nb, const mtp_batch* b, const int32_t* idx, int64_t n,
                                     int64_t* off, double* r, int32_t* type, int32_t* j, int64_t capacity,
                                     int64_t* total, void* stream) {
  return guarded([&] {
    if (!nb || !b || !off || !total || (n > 0 && !idx)) throw Fail{MTP_ERR_ARG, "null argument"};
    if (n < 0) throw Fail{MTP_ERR_ARG, "negative count"};
    DevBuf tmp;
    const int64_t t = run_extract(nb, b, idx, n, off, r, type, j, capacity, tmp, as_stream(stream));
    MTP_CUDA(cudaStreamSynchronize(as_stream(stream)));
    tmp.release();
    *total = t;
    if (t > capacity) throw Fail{MTP_ERR_CAPACITY, "extraction needs " + std::to_string(t) + " neighbor slots"};
  });
}

mtp_status mtp_cut_clusters(const mtp_batch* b, const int64_t* centers, int64_t n, double radius, int64_t* off,
                            double* pos, int32_t* type, int64_t* src, int64_t capacity, int64_t* total,
                            void* stream) {
  return guarded([&] {
    if (!b || !off || !total || (n > 0 && !centers)) throw Fail{MTP_ERR_ARG, "null argument"};
    if (n < 0 || capacity < 0) throw Fail{MTP_ERR_ARG, "negative count"};
    if (!(radius > 0.0) || !std::isfinite(radius)) throw Fail{MTP_ERR_ARG, "radius must be positive"};
    if (b->n_cfg <= 0 || !b->atom_offset || !b->pos || !b->type || !b->cell || !b->pbc)
      throw Fail{MTP_ERR_ARG, "incomplete batch"};
    const int64_t t = run_cut_clusters(b, centers, n, radius, off, pos, type, src, capacity, as_stream(stream));
    *total = t;
    if ((pos || type || src) && t > capacity)
      throw Fail{MTP_ERR_CAPACITY, "the clusters need " + std::to_string(t) + " atom slots"};
  });
}

mtp_status mtp_train_step(mtp_model* md, const mtp_batch* b, const mtp_nbr* nb, mtp_precision prec,
                          const double* E_ref, const double* F_ref, const double* W_ref, double w_e, double w_f,
                          double w_s, double* loss, double* grad, void* stream) {
  return guarded([&] {
    check_run(md, b, nb);
    if (!E_ref || !F_ref || !loss || !grad) throw Fail{MTP_ERR_ARG, "null argument"};
    if (w_s != 0.0 && !W_ref) throw Fail{MTP_ERR_ARG, "w_s != 0 needs W_ref"};
    if (w_e < 0 || w_f < 0 || w_s < 0) throw Fail{MTP_ERR_ARG, "weights must be non-negative"};
    cudaStream_t s = as_stream(stream);
    const bool fp64 = prec == MTP_FP64;
    const int64_t N = nb->n_atoms, P = nb->n_pairs, m = md->sched.n_params;
    const int n_cfg = static_cast<int>(nb->n_cfg);
    // pass 1: energies, forces, virials
    const size_t rsz = fp64 ? sizeof(double) : sizeof(float);
    md->ws_pair.ensure(std::max<int64_t>(P, 1) * 3 * rsz, s);
    // atom workspace: V, Wat(9), F(3), U(3)
    md->ws_atom.ensure(N * 16 * sizeof(double), s);
    double* V = md->ws_atom.as<double>();
    double* Wat = V + N;
    double* F = Wat + 9 * N;
    double* U = F + 3 * N;
    // config workspace: E, W, coef, S
    md->ws_misc.ensure(static_cast<size_t>(n_cfg) * 20 * sizeof(double) + 64, s);
    double* E = md->ws_misc.as<double>();
    double* W = E + n_cfg;
    double* coef = W + 9 * n_cfg;
    double* Sc = coef + n_cfg;
    SiteOutputs o;
    o.V = V; o.Wat = Wat; o.G = md->ws_pair.p;
    run_sites(md, b, nb, fp64, o, false, nullptr, s);
    run_forces(nb, fp64, o.G, F, s);
    run_config_sums(nb, V, Wat, E, W, md->ws_red, s);
    run_train_prep(nb, n_cfg, E, F, W, E_ref, F_ref, W_ref, w_e, w_f, w_s, coef, U, Sc, loss, md->ws_red, s);
    // pass 2: tangent of the parameter rows (forward-over-reverse), accumulated per warp
    SiteOutputs t;
    t.U = U;
    t.Scfg = Sc;
    t.coef = coef;
    const int rows_per_block = 4;
    int dev = 0, nsm = 0;
    MTP_CUDA(cudaGetDevice(&dev));
    MTP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int gmax = nsm * 4;
    const size_t part_bytes = static_cast<size_t>(gmax) * rows_per_block * m * sizeof(double);
    md->ws_rows.ensure(part_bytes, s);
    MTP_CUDA(cudaMemsetAsync(md->ws_rows.p, 0, part_bytes, s));
    t.grad_part = md->ws_rows.as<double>();
    int used = gmax;
    run_sites(md, b, nb, fp64, t, true, &used, s);
    run_sum_rows(t.grad_part, used * rows_per_block, m, grad, s);
  });
}

}  // extern "C"
