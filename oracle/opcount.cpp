// opcount.cpp -- op-counting build of the oracle.
//
// TEST INFRASTRUCTURE ONLY (like the rest of oracle/): it pins the
// arithmetic count per zone update that the benchmark's roofline divides by;
// nothing in the product path loads it.
//
// oracle.c is compiled here a second time, as C++, with every `double`
// replaced by `cdouble`: a value type holding one double that performs the
// same IEEE operation and adds one to a counter per +, -, *, / and sqrt
// (and, kept apart, per min/max, absolute value and comparison, which are
// not counted as flops).  The counters are kept per step of the scheme,
// which oracle.c marks with OR_STEP(k) at the start of each unit of work:
//   0 primitives of one cell            3 conservative update of one cell
//   1 slopes, predictor, face states    4 positivity check of a new cell
//     of one cell                       5 CFL signal speed of one cell
//   2 HLLC flux through one face
// so that ops per unit = ops attributed to the step / units opened.  The
// arithmetic itself is unchanged (same operations, same order, no
// contraction), so the counted run gives the normal oracle's results.
// Built single-threaded (no OpenMP): the counters are plain globals.

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

namespace opc {

enum Kind { ADD, SUB, MUL, DIV, SQRT, MINMAX, ABS, CMP, NKIND };
constexpr int kSteps = 7;   // steps 0..5, and 6 = outside any marked unit
unsigned long long g_ops[kSteps][NKIND];
unsigned long long g_units[kSteps];
int g_step = 6;

inline void tick(Kind k) { ++g_ops[g_step][k]; }

}  // namespace opc

struct cdouble {
  double v;
  cdouble() = default;
  constexpr cdouble(double x) : v(x) {}
  constexpr cdouble(float x) : v(x) {}
  constexpr cdouble(int x) : v(x) {}
  constexpr cdouble(long x) : v(double(x)) {}
  constexpr cdouble(long long x) : v(double(x)) {}
  constexpr cdouble(unsigned x) : v(x) {}
  constexpr cdouble(unsigned long x) : v(double(x)) {}
  explicit operator double() const { return v; }
  explicit operator int() const { return int(v); }
  explicit operator long() const { return long(v); }
  explicit operator long long() const { return (long long)v; }
  explicit operator bool() const { return v != 0.0; }
  cdouble &operator+=(cdouble o) { opc::tick(opc::ADD); v = v + o.v; return *this; }
  cdouble &operator-=(cdouble o) { opc::tick(opc::SUB); v = v - o.v; return *this; }
  cdouble &operator*=(cdouble o) { opc::tick(opc::MUL); v = v * o.v; return *this; }
  cdouble &operator/=(cdouble o) { opc::tick(opc::DIV); v = v / o.v; return *this; }
  cdouble operator-() const { return cdouble(-v); }   // sign flip: exact, not counted
  cdouble operator+() const { return *this; }
};

inline cdouble operator+(cdouble a, cdouble b) { opc::tick(opc::ADD); return cdouble(a.v + b.v); }
inline cdouble operator-(cdouble a, cdouble b) { opc::tick(opc::SUB); return cdouble(a.v - b.v); }
inline cdouble operator*(cdouble a, cdouble b) { opc::tick(opc::MUL); return cdouble(a.v * b.v); }
inline cdouble operator/(cdouble a, cdouble b) { opc::tick(opc::DIV); return cdouble(a.v / b.v); }
#define OPC_CMP(op)                                                                   \
  inline bool operator op(cdouble a, cdouble b) { opc::tick(opc::CMP); return a.v op b.v; }
OPC_CMP(<) OPC_CMP(<=) OPC_CMP(>) OPC_CMP(>=) OPC_CMP(==) OPC_CMP(!=)
#undef OPC_CMP

inline cdouble sqrt(cdouble a) { opc::tick(opc::SQRT); return cdouble(std::sqrt(a.v)); }
inline cdouble fabs(cdouble a) { opc::tick(opc::ABS); return cdouble(std::fabs(a.v)); }
inline cdouble fmin(cdouble a, cdouble b) { opc::tick(opc::MINMAX); return cdouble(std::fmin(a.v, b.v)); }
inline cdouble fmax(cdouble a, cdouble b) { opc::tick(opc::MINMAX); return cdouble(std::fmax(a.v, b.v)); }
inline bool isnan(cdouble a) { return std::isnan(a.v); }
inline bool isfinite(cdouble a) { return std::isfinite(a.v); }

#define OR_STEP(k) (opc::g_step = (k), ++opc::g_units[(k)])
#define double cdouble
#include "oracle.c"
#undef double

extern "C" {

// Clears every counter.
void or_opcount_reset(void) {
  std::memset(opc::g_ops, 0, sizeof opc::g_ops);
  std::memset(opc::g_units, 0, sizeof opc::g_units);
  opc::g_step = 6;
}

// ops[step][kind] (7 x 8: kinds add, sub, mul, div, sqrt, min/max, abs,
// compare) and units[step] (7), step 6 being work outside any marked unit.
void or_opcount_get(unsigned long long *ops, unsigned long long *units) {
  std::memcpy(ops, opc::g_ops, sizeof opc::g_ops);
  std::memcpy(units, opc::g_units, sizeof opc::g_units);
}

// Ends the current unit: later arithmetic counts as outside any unit.
void or_opcount_close(void) { opc::g_step = 6; }

}  // extern "C"
