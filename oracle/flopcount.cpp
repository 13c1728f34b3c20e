/*
 * Flop-counting build of the FP64 oracle (TEST AND MEASUREMENT INFRASTRUCTURE
 * ONLY, like the oracle itself): cg_oracle.c compiled as C++ with every
 * `double` replaced by a value type that counts the floating-point additions
 * and subtractions, multiplications, divisions and square roots it performs,
 * attributed to the step of the method (the ORC_REGION marks of cg_oracle.c)
 * running at the time.  A division or a square root counts as one operation;
 * comparisons, absolute values, negations, minima and maxima are not counted.
 * The arithmetic and its order are the oracle's own (no contraction), so the
 * counts are the algorithmic operation counts of the method as the oracle
 * states it.  Single-threaded (no OpenMP).
 */
#include <cmath>
#include <cstdint>
#include <cstring>

namespace fc {
enum { ADD, MUL, DIV, SQRT, NOPS };
constexpr int kMaxRegions = 32;
static const char* names[kMaxRegions] = {"other"};
static int nregions = 1;
static unsigned long long counts[kMaxRegions][NOPS];
static int cur = 0;

static int region_id(const char* name) {
  for (int i = 0; i < nregions; ++i)
    if (!std::strcmp(names[i], name)) return i;
  if (nregions == kMaxRegions) return 0;
  names[nregions] = name;
  return nregions++;
}

struct Region {
  int prev;
  explicit Region(const char* name) : prev(cur) { cur = region_id(name); }
  ~Region() { cur = prev; }
};
}  // namespace fc

struct cdouble {
  double v;
  cdouble() = default;
  constexpr cdouble(double x) : v(x) {}
  operator double() const { return v; }
  cdouble& operator+=(cdouble o) { ++fc::counts[fc::cur][fc::ADD]; v += o.v; return *this; }
  cdouble& operator-=(cdouble o) { ++fc::counts[fc::cur][fc::ADD]; v -= o.v; return *this; }
  cdouble& operator*=(cdouble o) { ++fc::counts[fc::cur][fc::MUL]; v *= o.v; return *this; }
  cdouble& operator/=(cdouble o) { ++fc::counts[fc::cur][fc::DIV]; v /= o.v; return *this; }
  cdouble operator-() const { return cdouble(-v); }
};
static_assert(sizeof(cdouble) == sizeof(double), "layout of the oracle's structs must not change");

#define FC_BIN(op, k)                                                                              \
  inline cdouble operator op(cdouble a, cdouble b) { ++fc::counts[fc::cur][k]; return cdouble(a.v op b.v); } \
  inline cdouble operator op(cdouble a, double b) { ++fc::counts[fc::cur][k]; return cdouble(a.v op b); }    \
  inline cdouble operator op(double a, cdouble b) { ++fc::counts[fc::cur][k]; return cdouble(a op b.v); }    \
  inline cdouble operator op(cdouble a, int b) { ++fc::counts[fc::cur][k]; return cdouble(a.v op b); }       \
  inline cdouble operator op(int a, cdouble b) { ++fc::counts[fc::cur][k]; return cdouble(a op b.v); }
FC_BIN(+, fc::ADD)
FC_BIN(-, fc::ADD)
FC_BIN(*, fc::MUL)
FC_BIN(/, fc::DIV)
#undef FC_BIN

inline cdouble sqrt(cdouble a) { ++fc::counts[fc::cur][fc::SQRT]; return cdouble(std::sqrt(a.v)); }
inline cdouble fabs(cdouble a) { return cdouble(std::fabs(a.v)); }
inline bool isnan(cdouble a) { return std::isnan(a.v); }

#define ORC_REGION(name) fc::Region fc_region_(#name)
#define double cdouble
extern "C" {
#include "cg_oracle.c"
}
#undef double

extern "C" {
void fc_reset(void) { std::memset(fc::counts, 0, sizeof fc::counts); }
int fc_regions(void) { return fc::nregions; }
const char* fc_region_name(int i) { return i >= 0 && i < fc::nregions ? fc::names[i] : ""; }
/* counts of region i: additions, multiplications, divisions, square roots */
void fc_region_counts(int i, unsigned long long out[4]) {
  for (int k = 0; k < fc::NOPS; ++k) out[k] = (i >= 0 && i < fc::nregions) ? fc::counts[i][k] : 0;
}
}
