// TTM schedules of CP-ALS-QR: no tree, the standard dimension tree and the
// restructured dimension tree (Section 3.1; costs in Tables 1-6 and Cor. 1).
#pragma once
#include <cstdint>
#include <map>
#include <vector>

namespace cpqr {

enum { OP_TTM = 0, OP_UPDATE = 1, OP_FREE = 2 };

struct Op {
  int32_t kind, a, b, c;  // TTM: dst, src, k | UPDATE: n, leaf, 0 | FREE: id, 0, 0
};

struct Node {
  uint32_t free_mask;       // modes still of full size I_k
  std::vector<int64_t> ver; // per mode: version of Q_k contracted, -1 if free
};

// Generates the operations of each sweep.  Node 0 is X; node ids count up from 1.
class Schedule {
 public:
  Schedule(const std::vector<int64_t>& dims, int R, int tree);
  // Appends the operations of the next sweep to `out`.
  void next_sweep(std::vector<Op>& out);
  int64_t flops() const { return flops_; }
  int64_t full_ttms() const { return full_ttms_; }
  int N() const { return N_; }

 private:
  std::vector<int> free_list(uint32_t mask) const;
  std::vector<int64_t> node_dims(uint32_t mask) const;
  int64_t ttm_cost(uint32_t mask) const;
  bool valid(const Node& nd) const;
  std::vector<int64_t> others(int n) const;  // versions of every Q_k but Q_n
  bool is_noop(int n) const;                 // no other factor changed since n's last update
  int ttm(int src, int k, std::vector<Op>& out);
  void update(int n, int leaf, std::vector<Op>& out);
  void release(int id, std::vector<Op>& out);
  void release_all(std::vector<Op>& out);
  void chain(int src, int n, const std::vector<int>& order, std::vector<Op>& out);
  void standard(int src, int m, bool top, std::vector<Op>& out);
  std::vector<int> no_tree_chain(int n) const;
  int find_valid(uint32_t mask) const;

  std::vector<int64_t> dims_;
  int N_, R_, tree_;
  std::vector<int64_t> ver_;
  std::vector<std::vector<int64_t>> seen_;  // per mode: others(n) at its last update
  std::map<int, Node> nodes_;
  int next_id_ = 1;
  int sweep_ = 0;
  int64_t flops_ = 0;
  int64_t full_ttms_ = 0;
};

}  // namespace cpqr
