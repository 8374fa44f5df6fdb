// space.cu — host planning of the expanded feature space (§2.1, Eq. 2) and expression
// strings.  The plan lists, per level l and enabled operator, the section of ids that
// operator creates: unary operators act on the features new at level l-1; binary
// operators act on pairs of phi_{l-1} that are not both in phi_{l-2} (those pairs were
// already generated), symmetric ones (+, *, -) once per unordered pair, / in both
// orders.  From level 3 on, grammar NEW_X_PREV keeps only pairs with one operand new at
// level l-1 and the other from phi_{l-2}.
#include "common.cuh"

#include <cstdio>

namespace sg {

bool plan_space(int d, uint32_t ops, int rung, int grammar, Space& sp) {
    if (d < 1 || rung < 0 || rung > kMaxRung) return false;
    sp = Space{};
    sp.d = d;
    sp.rung = rung;
    sp.grammar = grammar;
    sp.phi[0] = d;
    int64_t next = d;
    for (int l = 1; l <= rung; ++l) {
        const int64_t P = sp.phi[l - 1];
        const int64_t Q = l >= 2 ? sp.phi[l - 2] : 0;
        const bool nxp = grammar == SISSO_GRAMMAR_NEW_X_PREV && l >= 3;
        for (int op = 0; op < kNumOps; ++op) {
            if (!((ops >> op) & 1u)) continue;
            Section s{};
            s.level = l; s.op = op; s.P = P; s.Q = Q;
            if (op <= DIV) {
                const int64_t pairs = nxp ? Q * (P - Q) : P * (P - 1) / 2 - Q * (Q - 1) / 2;
                const bool div = op == DIV;
                s.kind = nxp ? (div ? K_DIV_NXP : K_SYM_NXP) : (div ? K_DIV_EQ2 : K_SYM_EQ2);
                s.count = div ? 2 * pairs : pairs;
            } else {
                s.kind = K_UNARY;
                s.count = P - Q;
            }
            if (s.count <= 0) continue;
            s.base = next;
            next += s.count;
            sp.sec[sp.nsec++] = s;
        }
        sp.phi[l] = next;
    }
    return true;
}

static void expr_rec(const Space& sp, int64_t id, std::string& out) {
    int level, op; int64_t a, b;
    if (!decode(sp, id, level, op, a, b)) { out += "?"; return; }
    if (level == 0) { out += "x" + std::to_string(a + 1); return; }
    std::string ea, eb;
    expr_rec(sp, a, ea);
    if (b >= 0) expr_rec(sp, b, eb);
    switch (op) {
        case ADD: out += "(" + ea + "+" + eb + ")"; break;
        case SUB: out += "(" + ea + "-" + eb + ")"; break;
        case MUL: out += "(" + ea + "*" + eb + ")"; break;
        case DIV: out += "(" + ea + "/" + eb + ")"; break;
        case EXP: out += "exp(" + ea + ")"; break;
        case LOG: out += "log(" + ea + ")"; break;
        case SQRT: out += "sqrt(" + ea + ")"; break;
        case SQ: out += "(" + ea + ")^2"; break;
        case INV: out += "(" + ea + ")^-1"; break;
        case SIN: out += "sin(" + ea + ")"; break;
        case CUBE: out += "(" + ea + ")^3"; break;
        default: out += "exp(-" + ea + ")"; break;
    }
}

std::string feature_expr(const Space& sp, int64_t id) {
    std::string s;
    expr_rec(sp, id, s);
    return s;
}

sisso_status fail(sisso_ctx* c, sisso_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

sisso_status check_cuda(sisso_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return SISSO_OK;
    return fail(c, e == cudaErrorMemoryAllocation ? SISSO_ERR_OOM : SISSO_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

double event_ms(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
}

}  // namespace sg
