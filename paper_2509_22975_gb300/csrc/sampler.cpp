// Monte Carlo construction of the truncated basis F~ on host threads.
//
// Sec. "Subspace of the ground state": starting from seed states, each step
// applies every hopping term to every starting state of the step; a proposed
// state b is accepted with probability min(exp(-beta * E_U(b)), 1) where
// E_U(b) = sum_i U_i n_i,up n_i,dn (the Boltzmann-factor Eq., U_i per site);
// accepted states start the next step (already-present ones included: the
// paper's "revisit"), new ones join F~ until it holds n_target states.
//
// Choices the paper leaves open (fixed so that runs are reproducible):
//   draw(step, parent, hop) = f(f(f(f(seed + G) ^ step) ^ parent) ^ hop), f =
//   the SplitMix64 output function, G = its golden gamma;
//   accept iff (draw >> 11) * 2^-53 < p;  hop id = s*n*n + i*n + j for
//   c^dag_{i s} c_{j s};  an overshooting last step keeps the new states of
//   smallest f(f(f(seed + G) ^ ~0) ^ word) (ties: smaller word); the run also
//   ends after 64 steps without a new state or when a step accepts nothing.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <unordered_map>

#include "mcd_internal.h"

namespace mcd {
namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

inline uint64_t smix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct Hop {
  uint64_t flip;   // bits toggled in the 64-bit word
  uint64_t from;   // bit that must be set
  uint64_t to;     // bit that must be clear
  uint64_t id;     // s*n*n + i*n + j
};

template <class F>
void parallel_for(int nthreads, int64_t n, F&& f) {
  if (nthreads <= 1 || n < 4096) {
    f(0, int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  int64_t chunk = (n + nthreads - 1) / nthreads;
  for (int t = 0; t < nthreads; ++t) {
    int64_t a = t * chunk, b = std::min(n, a + chunk);
    if (a >= b) break;
    th.emplace_back([&, t, a, b] { f(t, a, b); });
  }
  for (auto& x : th) x.join();
}

// Merge sorted unique runs into one sorted unique vector.
std::vector<uint64_t> merge_unique(std::vector<std::vector<uint64_t>>& runs) {
  while (runs.size() > 1) {
    std::vector<std::vector<uint64_t>> next((runs.size() + 1) / 2);
    std::vector<std::thread> th;
    for (size_t k = 0; k + 1 < runs.size(); k += 2) {
      th.emplace_back([&, k] {
        auto& a = runs[k];
        auto& b = runs[k + 1];
        std::vector<uint64_t> m;
        m.reserve(a.size() + b.size());
        std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(m));
        next[k / 2].swap(m);
        std::vector<uint64_t>().swap(a);
        std::vector<uint64_t>().swap(b);
      });
    }
    if (runs.size() % 2) next.back().swap(runs.back());
    for (auto& x : th) x.join();
    runs.swap(next);
  }
  if (runs.empty()) return {};
  return std::move(runs[0]);
}

}  // namespace

double sector_size(int n, int n_up, int n_dn) {
  auto binom = [](int a, int b) {
    double r = 1;
    for (int k = 1; k <= b; ++k) r = r * (a - b + k) / k;
    return std::floor(r + 0.5);
  };
  return binom(n, n_up) * binom(n, n_dn);
}

int sample_basis(mcd_ctx* c, uint64_t seed, int64_t n_target, double beta,
                 const uint64_t* seeds, int64_t n_seed, int flags,
                 std::vector<uint64_t>& out) {
  const int n = c->n;
  const uint64_t half = (n == 32) ? 0xFFFFFFFFull : ((1ull << n) - 1);
  // hopping terms in id order: spin, then i, then j
  std::vector<Hop> hops;
  for (int s = 0; s < 2; ++s) {
    const int shift = (s == 0) ? n : 0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        if (i == j || c->t[size_t(i) * n + j] == 0.0) continue;
        Hop h;
        h.from = 1ull << (j + shift);
        h.to = 1ull << (i + shift);
        h.flip = h.from | h.to;
        h.id = uint64_t(s) * n * n + uint64_t(i) * n + j;
        hops.push_back(h);
      }
  }
  // acceptance probability by double-occupancy pattern, E_U summed in site order
  const bool uniform = [&] {
    for (int i = 1; i < n; ++i)
      if (c->U[i] != c->U[0]) return false;
    return true;
  }();
  auto energy_p = [&](uint64_t both) {
    double e = 0.0;
    for (int i = 0; i < n; ++i)
      if ((both >> i) & 1) e += c->U[i];
    double p = std::exp(-beta * e);
    return p < 1.0 ? p : 1.0;
  };
  std::vector<double> ptab;
  if (uniform) {
    ptab.resize(n + 1);
    for (int k = 0; k <= n; ++k) ptab[k] = energy_p(k >= 64 ? ~0ull : ((1ull << k) - 1));
  }

  // seeds
  std::vector<uint64_t> F(seeds, seeds + n_seed);
  std::sort(F.begin(), F.end());
  F.erase(std::unique(F.begin(), F.end()), F.end());
  for (uint64_t w : F) {
    if (n < 32 && (w >> (2 * n)) != 0) return fail(c, MCD_E_SECTOR, "seed word has bits above 2*n_sites");
    if (__builtin_popcountll(w >> n) != c->n_up || __builtin_popcountll(w & half) != c->n_dn)
      return fail(c, MCD_E_SECTOR, "seed word outside the (N_up, N_dn) sector");
  }
  if (int64_t(F.size()) > n_target) return fail(c, MCD_E_INVALID, "more seed states than n_target");

  int nth = c->sampler_threads > 0 ? c->sampler_threads
                                   : std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  const uint64_t key1 = smix(seed + kGamma);
  std::vector<uint64_t> frontier = F;
  uint64_t step = 0;
  int stagnant = 0;
  int status = MCD_OK;
  while (int64_t(F.size()) < n_target) {
    ++step;
    const uint64_t key2 = smix(key1 ^ step);
    std::vector<std::vector<uint64_t>> runs(nth);
    parallel_for(nth, int64_t(frontier.size()), [&](int t, int64_t a, int64_t b) {
      auto& acc = runs[t];
      for (int64_t k = a; k < b; ++k) {
        const uint64_t w = frontier[k];
        const uint64_t key3 = smix(key2 ^ w);
        for (const Hop& h : hops) {
          if (!(w & h.from) || (w & h.to)) continue;
          const uint64_t child = w ^ h.flip;
          const uint64_t r = smix(key3 ^ h.id);
          const uint64_t both = (child >> n) & child & half;
          const double p = uniform ? ptab[__builtin_popcountll(both)] : energy_p(both);
          const double u = double(r >> 11) * 0x1p-53;
          if (u < p) acc.push_back(child);
        }
      }
      std::sort(acc.begin(), acc.end());
      acc.erase(std::unique(acc.begin(), acc.end()), acc.end());
    });
    std::vector<uint64_t> accepted = merge_unique(runs);
    std::vector<uint64_t> fresh;
    std::set_difference(accepted.begin(), accepted.end(), F.begin(), F.end(),
                        std::back_inserter(fresh));
    const int64_t room = n_target - int64_t(F.size());
    if (int64_t(fresh.size()) > room) {
      const uint64_t kp = smix(key1 ^ ~0ull);
      std::vector<std::pair<uint64_t, uint64_t>> pr(fresh.size());
      for (size_t k = 0; k < fresh.size(); ++k) pr[k] = {smix(kp ^ fresh[k]), fresh[k]};
      std::nth_element(pr.begin(), pr.begin() + room, pr.end());
      fresh.resize(room);
      for (int64_t k = 0; k < room; ++k) fresh[k] = pr[k].second;
      std::sort(fresh.begin(), fresh.end());
    }
    const bool none_accepted = accepted.empty();
    std::vector<uint64_t> merged;
    merged.reserve(F.size() + fresh.size());
    std::merge(F.begin(), F.end(), fresh.begin(), fresh.end(), std::back_inserter(merged));
    F.swap(merged);
    stagnant = fresh.empty() ? stagnant + 1 : 0;
    if (flags & MCD_SAMPLE_NEW_ONLY)
      frontier.swap(fresh);
    else
      frontier.swap(accepted);
    if (int64_t(F.size()) >= n_target) break;
    if (none_accepted || frontier.empty() || stagnant >= 64) { status = MCD_W_SHORT; break; }
  }
  out.swap(F);
  return status;
}

}  // namespace mcd
