// TTM schedules (Section 3.1).  A TTM on a node with free modes F costs
// 2 * R * prod(dims of the node) flops (Section 3.4).
//
// * Standard dimension tree (Tables 1 and 4): the modes {0..m-1} of a node
//   split into {0..m-2} through a contraction of mode m-1, and into the leaf
//   m-1 through contractions of modes 0..m-2 - ascending at the top level of
//   an order >= 4 tree, descending otherwise.  Each sweep restarts from X.
// * Restructured tree: the first sweep is the standard tree and every node
//   stays cached while all Q_k it contracted are current.  Order 3 alternates
//   the two sweeps of Section 3.1 (A1 from the unused Y(1,3), then Y(2,3) from
//   X for A2 and A3; A2 from Y(2,3), then Y(1,3) from X for A1 and A3).  Order
//   4 sweeps 2 and 3 follow the structure counted in Table 5 (reusing Y(3,4),
//   Y(2,3,4), Y(1,3,4), Y(1,4)).  Every other sweep repeatedly picks, among the
//   modes not yet updated in the sweep whose update is not a no-op (a mode is a
//   no-op while no other factor changed since its last update), the cached
//   source whose contraction chain is cheapest (ties: lower mode, then the
//   lexicographically smaller free set, then the older node); the chain
//   contracts the modes already updated in the sweep first, then ascending.
// * No tree (Tables 3 and 6): each mode contracts X directly; order 3 uses the
//   cyclic predecessors, higher orders contract the last modes first for the
//   lower half of the modes and the first modes first for the upper half.
#include "schedule.h"

#include <algorithm>
#include <cassert>
#include <stdexcept>

namespace cpqr {

namespace {
struct Step {
  int n;
  uint32_t src_mask;
  std::vector<int> chain;
};
// Order-3 restructured sweeps 2 and 3, repeated with period 2 (0-based modes).
const std::vector<std::vector<Step>>& order3_steps() {
  static const std::vector<std::vector<Step>> s = {
      {{0, 0b101u, {2}}, {1, 0b111u, {0, 2}}, {2, 0b110u, {1}}},
      {{1, 0b110u, {2}}, {0, 0b111u, {1, 2}}, {2, 0b101u, {0}}},
  };
  return s;
}
// Order-4 restructured sweeps 2 and 3 (0-based modes).
const std::vector<std::vector<Step>>& order4_steps() {
  static const std::vector<std::vector<Step>> s = {
      {{2, 0b1100u, {3}}, {1, 0b1110u, {2, 3}}, {0, 0b1111u, {1, 2, 3}}, {3, 0b1001u, {0}}},
      {{0, 0b1001u, {3}}, {2, 0b1101u, {0, 3}}, {1, 0b1111u, {2, 0, 3}}, {3, 0b1010u, {1}}},
  };
  return s;
}
}  // namespace

Schedule::Schedule(const std::vector<int64_t>& dims, int R, int tree)
    : dims_(dims), N_((int)dims.size()), R_(R), tree_(tree), ver_(dims.size(), 0), seen_(dims.size()) {
  Node x;
  x.free_mask = (1u << N_) - 1u;
  x.ver.assign(N_, -1);
  nodes_[0] = x;
}

std::vector<int> Schedule::free_list(uint32_t mask) const {
  std::vector<int> f;
  for (int k = 0; k < N_; ++k)
    if (mask & (1u << k)) f.push_back(k);
  return f;
}

std::vector<int64_t> Schedule::node_dims(uint32_t mask) const {
  std::vector<int64_t> d(N_);
  for (int k = 0; k < N_; ++k) d[k] = (mask & (1u << k)) ? dims_[k] : R_;
  return d;
}

int64_t Schedule::ttm_cost(uint32_t mask) const {
  int64_t p = 2 * (int64_t)R_;
  for (int64_t v : node_dims(mask)) p *= v;
  return p;
}

std::vector<int64_t> Schedule::others(int n) const {
  std::vector<int64_t> v;
  for (int k = 0; k < N_; ++k)
    if (k != n) v.push_back(ver_[k]);
  return v;
}

bool Schedule::is_noop(int n) const { return !seen_[n].empty() && seen_[n] == others(n); }

bool Schedule::valid(const Node& nd) const {
  for (int k = 0; k < N_; ++k)
    if (nd.ver[k] >= 0 && nd.ver[k] != ver_[k]) return false;
  return true;
}

int Schedule::ttm(int src, int k, std::vector<Op>& out) {
  const Node& s = nodes_.at(src);
  if (!(s.free_mask & (1u << k))) throw std::logic_error("ttm on a contracted mode");
  flops_ += ttm_cost(s.free_mask);
  if (src == 0) ++full_ttms_;
  Node d;
  d.free_mask = s.free_mask & ~(1u << k);
  d.ver = s.ver;
  d.ver[k] = ver_[k];
  int id = next_id_++;
  nodes_[id] = d;
  out.push_back({OP_TTM, id, src, k});
  return id;
}

void Schedule::release(int id, std::vector<Op>& out) {
  nodes_.erase(id);
  out.push_back({OP_FREE, id, 0, 0});
}

void Schedule::release_all(std::vector<Op>& out) {
  std::vector<int> ids;
  for (auto& kv : nodes_)
    if (kv.first != 0) ids.push_back(kv.first);
  for (int id : ids) release(id, out);
}

void Schedule::update(int n, int leaf, std::vector<Op>& out) {
  const Node& l = nodes_.at(leaf);
  if (l.free_mask != (1u << n) || !valid(l)) throw std::logic_error("invalid leaf");
  out.push_back({OP_UPDATE, n, leaf, 0});
  seen_[n] = others(n);
  ++ver_[n];
  release(leaf, out);
  std::vector<int> stale;
  for (auto& kv : nodes_)
    if (kv.first != 0 && kv.second.ver[n] >= 0) stale.push_back(kv.first);
  for (int id : stale) release(id, out);
}

void Schedule::chain(int src, int n, const std::vector<int>& order, std::vector<Op>& out) {
  int cur = src;
  for (int k : order) cur = ttm(cur, k, out);
  update(n, cur, out);
}

std::vector<int> Schedule::no_tree_chain(int n) const {
  std::vector<int> c;
  if (N_ == 3) {
    c.push_back((n + 2) % 3);
    c.push_back((n + 1) % 3);
  } else if (n < N_ / 2) {
    for (int k = N_ - 1; k >= 0; --k)
      if (k != n) c.push_back(k);
  } else {
    for (int k = 0; k < N_; ++k)
      if (k != n) c.push_back(k);
  }
  return c;
}

void Schedule::standard(int src, int m, bool top, std::vector<Op>& out) {
  if (m == 1) {
    update(0, src, out);
    return;
  }
  int left = ttm(src, m - 1, out);
  standard(left, m - 1, false, out);
  std::vector<int> order;
  if (top && N_ >= 4) {
    for (int k = 0; k <= m - 2; ++k) order.push_back(k);
  } else {
    for (int k = m - 2; k >= 0; --k) order.push_back(k);
  }
  chain(src, m - 1, order, out);
}

int Schedule::find_valid(uint32_t mask) const {
  for (auto& kv : nodes_)
    if (kv.second.free_mask == mask && valid(kv.second)) return kv.first;
  throw std::logic_error("no valid cached node for a tabulated step");
}

void Schedule::next_sweep(std::vector<Op>& out) {
  const int s = sweep_++;
  if (tree_ == 0) {
    for (int n = 0; n < N_; ++n) {
      chain(0, n, no_tree_chain(n), out);
      release_all(out);
    }
    return;
  }
  if (tree_ == 1 || s == 0) {
    standard(0, N_, true, out);
    if (tree_ == 1) release_all(out);
    return;
  }
  if (N_ == 3) {
    for (const Step& st : order3_steps()[(s - 1) % 2]) chain(find_valid(st.src_mask), st.n, st.chain, out);
    return;
  }
  if (N_ == 4 && (s == 1 || s == 2)) {
    for (const Step& st : order4_steps()[s - 1]) chain(find_valid(st.src_mask), st.n, st.chain, out);
    return;
  }
  uint32_t done = 0;
  for (int step = 0; step < N_; ++step) {
    bool have = false;
    int64_t best_cost = 0;
    int best_n = 0, best_id = 0;
    std::vector<int> best_free, best_chain;
    for (int n = 0; n < N_; ++n) {
      if ((done & (1u << n)) || is_noop(n)) continue;
      for (auto& kv : nodes_) {
        const Node& nd = kv.second;
        if (!(nd.free_mask & (1u << n)) || !valid(nd)) continue;
        std::vector<int> updated, rest;
        for (int k : free_list(nd.free_mask)) {
          if (k == n) continue;
          if (done & (1u << k)) updated.push_back(k);
          else rest.push_back(k);
        }
        std::vector<int> ch = updated;
        ch.insert(ch.end(), rest.begin(), rest.end());
        std::vector<int64_t> d = node_dims(nd.free_mask);
        int64_t cost = 0;
        for (int k : ch) {
          int64_t p = 2 * (int64_t)R_;
          for (int64_t v : d) p *= v;
          cost += p;
          d[k] = R_;
        }
        std::vector<int> fl = free_list(nd.free_mask);
        bool better = !have || cost < best_cost || (cost == best_cost && n < best_n) ||
                      (cost == best_cost && n == best_n && fl < best_free);
        if (better) {
          have = true;
          best_cost = cost;
          best_n = n;
          best_id = kv.first;
          best_free = fl;
          best_chain = ch;
        }
      }
    }
    if (!have) throw std::logic_error("no valid source");
    chain(best_id, best_n, best_chain, out);
    done |= 1u << best_n;
  }
}

}  // namespace cpqr
