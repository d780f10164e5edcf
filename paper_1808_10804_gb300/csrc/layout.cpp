// Canonical block layouts of U(1)- and Z2-symmetric tensors (Sec. 2).
//
// A block is one sector per leg; it is allowed iff sum_i flow_i q_i = 0
// (no global charge shift, Sec. 2), for Z2 modulo 2.  Blocks are kept in lexicographic order
// of their per-leg sector indices (leg 0 most significant), each stored
// dense row-major, back to back.  Layouts are interned per context by their
// structure, so equal structures are the same object and plans keyed by
// layout pointers are reused across calls.
#include <algorithm>
#include <functional>
#include <numeric>
#include <sstream>

#include "bst_internal.h"

namespace bst {

void Leg::finish() {
  off.assign(q.size() + 1, 0);
  for (size_t i = 0; i < q.size(); ++i) off[i + 1] = off[i] + d[i];
  dim = off.back();
}

int Leg::find(int charge) const {
  auto it = std::lower_bound(q.begin(), q.end(), charge);
  if (it == q.end() || *it != charge) return -1;
  return int(it - q.begin());
}

int64_t Layout::block_of(const int32_t* s) const {
  auto it = index.find(pack(s, rank));
  return it == index.end() ? -1 : it->second;
}

static std::string layout_key(int group, const std::vector<Leg>& legs) {
  std::ostringstream os;
  os << group << "|";
  for (auto& l : legs) {
    os << l.flow << ":";
    for (size_t i = 0; i < l.q.size(); ++i) os << l.q[i] << "x" << l.d[i] << ",";
    os << ";";
  }
  return os.str();
}

// Depth-first enumeration of allowed sector tuples in lexicographic order,
// pruned with the reachable range of the remaining partial sums.
static void enum_blocks(const std::vector<Leg>& legs, std::vector<int32_t>& out, int group) {
  const int r = int(legs.size());
  if (group == BST_Z2) {
    // parities: every tuple whose charges add up to an even number
    std::vector<int32_t> cur(r);
    std::function<void(int, int64_t)> rec = [&](int i, int64_t sum) {
      if (i == r) {
        if (cnorm(group, sum) == 0) out.insert(out.end(), cur.begin(), cur.end());
        return;
      }
      for (int s = 0; s < int(legs[i].q.size()); ++s) {
        cur[i] = s;
        rec(i + 1, sum + legs[i].q[s]);
      }
    };
    rec(0, 0);
    return;
  }
  std::vector<int64_t> lo(r + 1, 0), hi(r + 1, 0);
  for (int i = r - 1; i >= 0; --i) {
    int64_t a = int64_t(legs[i].flow) * legs[i].q.front();
    int64_t b = int64_t(legs[i].flow) * legs[i].q.back();
    lo[i] = lo[i + 1] + std::min(a, b);
    hi[i] = hi[i + 1] + std::max(a, b);
  }
  std::vector<int32_t> cur(r);
  std::function<void(int, int64_t)> rec = [&](int i, int64_t sum) {
    if (i == r) {
      if (sum == 0) out.insert(out.end(), cur.begin(), cur.end());
      return;
    }
    if (sum + lo[i] > 0 || sum + hi[i] < 0) return;
    for (int s = 0; s < int(legs[i].q.size()); ++s) {
      cur[i] = s;
      rec(i + 1, sum + int64_t(legs[i].flow) * legs[i].q[s]);
    }
  };
  rec(0, 0);
}

Layout* make_layout(Ctx* ctx, int group, const std::vector<Leg>& legs_in) {
  BST_REQUIRE(group == BST_U1 || group == BST_SU2 || group == BST_Z2, BST_E_ARG,
              "group must be BST_U1, BST_SU2 or BST_Z2");
  BST_REQUIRE(!legs_in.empty() && legs_in.size() <= kMaxRank, BST_E_ARG, "rank must be 1..8");
  std::vector<Leg> legs = legs_in;
  for (auto& l : legs) {
    BST_REQUIRE(l.flow == 1 || l.flow == -1, BST_E_ARG, "flow must be +1 or -1");
    BST_REQUIRE(!l.q.empty() && l.q.size() == l.d.size() && l.q.size() < 255, BST_E_ARG,
                "a leg needs 1..254 sectors");
    for (size_t i = 0; i < l.q.size(); ++i) {
      BST_REQUIRE(l.d[i] > 0, BST_E_ARG, "degeneracies must be positive");
      if (i) BST_REQUIRE(l.q[i] > l.q[i - 1], BST_E_ARG, "charges must be strictly ascending");
      if (group == BST_SU2) BST_REQUIRE(l.q[i] >= 0 && l.q[i] <= 64, BST_E_ARG, "SU(2) labels 2j must be 0..64");
      if (group == BST_Z2) BST_REQUIRE(l.q[i] == 0 || l.q[i] == 1, BST_E_ARG, "Z2 charges must be 0 or 1");
    }
    l.finish();
  }
  std::string key = layout_key(group, legs);
  std::lock_guard<std::mutex> g(ctx->mu);
  auto it = ctx->interned.find(key);
  if (it != ctx->interned.end()) {
    it->second->refs++;
    return it->second;
  }
  auto* L = new Layout();
  L->ctx = ctx;
  L->id = ctx->next_id++;
  L->group = group;
  L->rank = int(legs.size());
  L->legs = legs;
  L->key = key;
  if (group == BST_SU2) {
    L->ntree = su2_ntree(legs);
    su2_enum_blocks(legs, L->sect, L->tree);
  } else {
    enum_blocks(legs, L->sect, group);
  }
  L->nblocks = int64_t(L->sect.size()) / L->rank;
  L->offset.resize(L->nblocks);
  L->shape.resize(L->nblocks * L->rank);
  int64_t off = 0;
  for (int64_t b = 0; b < L->nblocks; ++b) {
    int64_t n = 1;
    for (int i = 0; i < L->rank; ++i) {
      int64_t e = legs[i].d[L->sect[b * L->rank + i]];
      L->shape[b * L->rank + i] = e;
      n *= e;
    }
    BST_REQUIRE(n < (int64_t(1) << 31), BST_E_SHAPE, "block larger than 2^31 elements");
    L->offset[b] = off;
    off += n;
    L->index.emplace(Layout::pack(&L->sect[b * L->rank], L->rank), b);  // first block of a tuple
  }
  L->nnz = off;
  L->refs = 2;  // one for the caller, one for the intern table
  ctx->interned[key] = L;
  return L;
}

void retain(Layout* l) {
  if (l) l->refs++;
}

void release(Layout* l) {
  if (!l) return;
  // The intern table keeps one reference until the context goes away.
  if (--l->refs == 0) delete l;
}

std::vector<std::vector<int32_t>> enum_configs(const std::vector<const Leg*>& legs, int64_t target, int group) {
  // all sector tuples over `legs` with sum_i flow_i q_i == target (Z2: of the
  // same parity), lexicographic
  std::vector<std::vector<int32_t>> out;
  const int r = int(legs.size());
  if (r == 0) {
    if (cnorm(group, target) == 0) out.push_back({});
    return out;
  }
  if (group == BST_Z2) {
    std::vector<int32_t> cur(r);
    std::function<void(int, int64_t)> rec = [&](int i, int64_t sum) {
      if (i == r) {
        if (cnorm(group, sum - target) == 0) out.push_back(cur);
        return;
      }
      for (int s = 0; s < int(legs[i]->q.size()); ++s) {
        cur[i] = s;
        rec(i + 1, sum + legs[i]->q[s]);
      }
    };
    rec(0, 0);
    return out;
  }
  std::vector<int64_t> lo(r + 1, 0), hi(r + 1, 0);
  for (int i = r - 1; i >= 0; --i) {
    int64_t a = int64_t(legs[i]->flow) * legs[i]->q.front();
    int64_t b = int64_t(legs[i]->flow) * legs[i]->q.back();
    lo[i] = lo[i + 1] + std::min(a, b);
    hi[i] = hi[i + 1] + std::max(a, b);
  }
  std::vector<int32_t> cur(r);
  std::function<void(int, int64_t)> rec = [&](int i, int64_t sum) {
    if (i == r) {
      if (sum == target) out.push_back(cur);
      return;
    }
    if (sum + lo[i] > target || sum + hi[i] < target) return;
    for (int s = 0; s < int(legs[i]->q.size()); ++s) {
      cur[i] = s;
      rec(i + 1, sum + int64_t(legs[i]->flow) * legs[i]->q[s]);
    }
  };
  rec(0, 0);
  return out;
}

// Fused leg (Sec. 3.2, merging legs): flow of the first member, charge
// flow_0 * sum_i flow_i q_i (Z2: its parity), sectors ascending, member
// tuples ascending lexicographically inside a sector, inner index row-major
// over members.
Leg fuse_legs(const std::vector<Leg>& legs, std::vector<std::vector<int32_t>>* tuples, int group) {
  const int f0 = legs[0].flow;
  std::map<int64_t, std::vector<std::vector<int32_t>>> byq;
  std::vector<int32_t> cur(legs.size());
  std::function<void(size_t, int64_t)> rec = [&](size_t i, int64_t sum) {
    if (i == legs.size()) {
      byq[cnorm(group, sum * f0)].push_back(cur);
      return;
    }
    for (int s = 0; s < int(legs[i].q.size()); ++s) {
      cur[i] = s;
      rec(i + 1, sum + int64_t(legs[i].flow) * legs[i].q[s]);
    }
  };
  rec(0, 0);
  Leg out;
  out.flow = f0;
  if (tuples) tuples->clear();
  for (auto& kv : byq) {
    int64_t deg = 0;
    for (auto& t : kv.second) {
      int64_t n = 1;
      for (size_t i = 0; i < legs.size(); ++i) n *= legs[i].d[t[i]];
      deg += n;
    }
    out.q.push_back(int(kv.first));
    out.d.push_back(deg);
  }
  if (tuples) {
    // flattened: for each sector, the tuples in order (sector boundaries
    // are recovered from the degeneracies)
    for (auto& kv : byq)
      for (auto& t : kv.second) tuples->push_back(t);
  }
  out.finish();
  return out;
}

}  // namespace bst
