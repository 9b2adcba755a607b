// mk_compile.cpp -- formula text -> slot-annotated postfix program (host).
//
// The formula language is the one of Sec. 2 (T, F, p_i, negation,
// conjunction, disjunction, implication, box, diamond); the program is the
// bitmask recurrence of Sec. 3 (Thm. 1) laid out as straight-line postfix
// code, the compiled-program form the corpus scan of Sec. 4 interprets.
//
// Differences from the paper's 48-slot semantic stack (Sec. 4, "272 bytes of
// thread-local storage"): the program runs on an accumulator plus a stack
// whose depth is minimised at compile time (Sethi-Ullman order, variable
// operands fused into the binary instruction), so random 64-node formulas
// need at most three saved truth sets and the device keeps the accumulator
// in registers and the few saved sets in shared memory.
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "mk.h"

namespace {

enum Kind { TOP, BOT, VAR, NOT, AND, OR, IMP, IFF, BOX, DIA };

struct Node {
    Kind kind;
    int var = 0;
    int a = -1, b = -1;
    bool neg = false;          // VAR only: the negated atom
};

struct Tree {
    std::vector<Node> nodes;
    int add(Kind k, int a = -1, int b = -1, int var = 0, bool neg = false) {
        nodes.push_back(Node{k, var, a, b, neg});
        return (int)nodes.size() - 1;
    }
};

// ----------------------------------------------------------------- parser

class Parser {
  public:
    Parser(const char *s, Tree &t) : s_(s), t_(t) {}
    int parse_all(int &root) {
        root = iff();
        ws();
        if (!err_ && s_[i_] != 0) fail();
        return err_ ? MK_E_SYNTAX : (bad_var_ ? MK_E_VARS : MK_OK);
    }
    int error_pos() const { return err_ ? err_pos_ : -1; }
    int nvars() const { return nvars_; }

  private:
    const char *s_;
    Tree &t_;
    int i_ = 0;
    bool err_ = false, bad_var_ = false;
    int err_pos_ = -1, nvars_ = 0;

    void fail() {
        if (!err_) { err_ = true; err_pos_ = i_; }
    }
    void ws() {
        while (s_[i_] == ' ' || s_[i_] == '\t' || s_[i_] == '\n' || s_[i_] == '\r') i_++;
    }
    static bool alnum(char c) {
        return (c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z') || (c >= '0' && c <= '9') || c == '_';
    }
    bool eat(const char *tok) {
        ws();
        size_t L = std::strlen(tok);
        if (std::strncmp(s_ + i_, tok, L) != 0) return false;
        if (alnum(tok[0]) && alnum(s_[i_ + L])) return false;
        i_ += (int)L;
        return true;
    }
    int iff() {
        int e = imp();
        while (!err_ && eat("<->")) e = t_.add(IFF, e, imp());
        return e;
    }
    int imp() {
        int e = disj();
        ws();
        if (!err_ && std::strncmp(s_ + i_, "<->", 3) != 0 && eat("->")) return t_.add(IMP, e, imp());
        return e;
    }
    int disj() {
        int e = conj();
        while (!err_ && (eat("|") || eat("or"))) e = t_.add(OR, e, conj());
        return e;
    }
    int conj() {
        int e = unary();
        while (!err_ && (eat("&") || eat("and"))) e = t_.add(AND, e, unary());
        return e;
    }
    int unary() {
        if (err_) return 0;
        if (eat("~") || eat("!") || eat("not")) return t_.add(NOT, unary());
        if (eat("[]") || eat("box")) return t_.add(BOX, unary());
        if (eat("<>") || eat("dia")) return t_.add(DIA, unary());
        if (eat("(")) {
            int e = iff();
            if (!eat(")")) fail();
            return e;
        }
        if (eat("T") || eat("true")) return t_.add(TOP);
        if (eat("F") || eat("false")) return t_.add(BOT);
        ws();
        char c = s_[i_];
        int var = -1;
        if (c == 'p' && s_[i_ + 1] >= '0' && s_[i_ + 1] <= '9') {
            int j = i_ + 1;
            long v = 0;
            while (s_[j] >= '0' && s_[j] <= '9' && v < 1000) v = v * 10 + (s_[j++] - '0');
            if (alnum(s_[j])) { fail(); return 0; }
            var = (int)v;
            i_ = j;
        } else if ((c == 'p' || c == 'q' || c == 'r' || c == 's') && !alnum(s_[i_ + 1])) {
            var = c == 'p' ? 0 : c == 'q' ? 1 : c == 'r' ? 2 : 3;
            i_++;
        } else {
            fail();
            return 0;
        }
        if (var >= MK_MAX_VARS) bad_var_ = true;
        if (var + 1 > nvars_) nvars_ = var + 1;
        return t_.add(VAR, -1, -1, var);
    }
};

// ---------------------------------------------------------- statistics

int count_nodes(const Tree &t, int id) {
    const Node &n = t.nodes[id];
    int c = 1;
    if (n.a >= 0) c += count_nodes(t, n.a);
    if (n.b >= 0) c += count_nodes(t, n.b);
    return c;
}

int modal_depth(const Tree &t, int id) {
    const Node &n = t.nodes[id];
    int d = 0;
    if (n.a >= 0) d = modal_depth(t, n.a);
    if (n.b >= 0) {
        int e = modal_depth(t, n.b);
        if (e > d) d = e;
    }
    return d + ((n.kind == BOX || n.kind == DIA) ? 1 : 0);
}

// ---------------------------------------------------- constant folding
// Each rule is a propositional or normal-modal identity on truth sets:
// []W = W and <>{} = {} (Lemma 1 with t = full / t = 0).

bool is_const(const Tree &t, int id, Kind k) { return t.nodes[id].kind == k; }

int fold(Tree &t, int id) {
    Node n = t.nodes[id];
    if (n.a >= 0) n.a = fold(t, n.a);
    if (n.b >= 0) n.b = fold(t, n.b);
    t.nodes[id] = n;
    auto top = [&](int x) { return is_const(t, x, TOP); };
    auto bot = [&](int x) { return is_const(t, x, BOT); };
    switch (n.kind) {
    case NOT:
        if (top(n.a)) return t.add(BOT);
        if (bot(n.a)) return t.add(TOP);
        return id;
    case AND:
        if (bot(n.a) || bot(n.b)) return t.add(BOT);
        if (top(n.a)) return n.b;
        if (top(n.b)) return n.a;
        return id;
    case OR:
        if (top(n.a) || top(n.b)) return t.add(TOP);
        if (bot(n.a)) return n.b;
        if (bot(n.b)) return n.a;
        return id;
    case IMP:
        if (bot(n.a) || top(n.b)) return t.add(TOP);
        if (top(n.a)) return n.b;
        if (bot(n.b)) return fold(t, t.add(NOT, n.a));
        return id;
    case IFF:
        if (top(n.a)) return n.b;
        if (top(n.b)) return n.a;
        if (bot(n.a)) return fold(t, t.add(NOT, n.b));
        if (bot(n.b)) return fold(t, t.add(NOT, n.a));
        return id;
    case BOX:
        if (top(n.a)) return t.add(TOP);
        return id;
    case DIA:
        if (bot(n.a)) return t.add(BOT);
        return id;
    default:
        return id;
    }
}

// ------------------------------------------------- negation normal form
// Negations are pushed to the atoms (Sec. 2's clauses make each rule an
// identity on truth sets): ~~a = a, De Morgan for & and |, ~(a -> b) =
// a & ~b, and the duality ~[]a = <>~a, ~<>a = []~a (Lemma 1: the
// complement of {w : succ[w] subset of t} is {w : succ[w] meets W \ t}).
// A negated atom is a leaf of its own (the LDNV / *_NV instructions); a
// negated biconditional keeps its NOT.  No rule adds an instruction, and
// the tree shape (so the stack depth) is unchanged.
int nnf(Tree &t, int id, bool neg) {
    const Node n = t.nodes[id];
    switch (n.kind) {
    case TOP: return neg ? t.add(BOT) : id;
    case BOT: return neg ? t.add(TOP) : id;
    case VAR: return neg ? t.add(VAR, -1, -1, n.var, !n.neg) : id;
    case NOT: return nnf(t, n.a, !neg);
    case AND: {
        const int a = nnf(t, n.a, neg), b = nnf(t, n.b, neg);
        return t.add(neg ? OR : AND, a, b);
    }
    case OR: {
        const int a = nnf(t, n.a, neg), b = nnf(t, n.b, neg);
        return t.add(neg ? AND : OR, a, b);
    }
    case IMP: {
        const int a = nnf(t, n.a, false), b = nnf(t, n.b, neg);
        return t.add(neg ? AND : IMP, a, b);
    }
    case IFF: {
        const int e = t.add(IFF, nnf(t, n.a, false), nnf(t, n.b, false));
        return neg ? t.add(NOT, e) : e;
    }
    case BOX: return t.add(neg ? DIA : BOX, nnf(t, n.a, neg));
    case DIA: return t.add(neg ? BOX : DIA, nnf(t, n.a, neg));
    }
    return id;
}

// ------------------------------------------------------------ codegen
// Accumulator machine (mk.h): a subtree is evaluated into A; for a binary
// node whose operands are both compound, the operand needing the deeper
// stack is evaluated first, pushed at the current depth, and the other one
// evaluated above it (Sethi-Ullman order, so the stack depth is minimal).
// A variable operand of a binary node is fused into the instruction.

struct Gen {
    const Tree &t;
    std::vector<uint8_t> code;
    int max_depth = 0;
    int n_modal = 0, n_bool = 0;
    bool overflow = false;

    explicit Gen(const Tree &tr) : t(tr) {}

    bool is_var(int id) const { return t.nodes[id].kind == VAR; }
    bool fusable(const Node &n) const { return n.kind != IFF && (is_var(n.b) || is_var(n.a)); }

    // stack entries needed to evaluate node id
    int depth(int id) const {
        const Node &n = t.nodes[id];
        switch (n.kind) {
        case TOP: case BOT: case VAR: return 0;
        case NOT: case BOX: case DIA: return depth(n.a);
        default: {
            if (fusable(n)) return depth(is_var(n.b) ? n.a : n.b);
            int x = depth(n.a), y = depth(n.b);
            int first = x >= y ? x : y, second = x >= y ? y : x;
            int d = second + 1;
            return first > d ? first : d;
        }
        }
    }

    void emit(int op, int operand) {
        code.push_back((uint8_t)(op | (operand << 5)));
        const bool modal = op == MK_OP_BOX || op == MK_OP_DIA || op >= MK_OP_BOX_V;
        if (modal) n_modal++;
        // negating and binary steps (LDNV and the *_NV modal forms negate)
        if (op == MK_OP_NOT || (op >= MK_OP_AND_S && op < MK_OP_BOX_V) || op == MK_OP_BOX_NV ||
            op == MK_OP_DIA_NV)
            n_bool++;
    }

    // binary node with a (possibly negated) variable operand: the variable
    // is on the left (var_left) or the right
    static int var_op(Kind k, bool var_left, bool neg) {
        switch (k) {
        case AND: return neg ? MK_OP_AND_NV : MK_OP_AND_V;
        case OR: return neg ? MK_OP_OR_NV : MK_OP_OR_V;
        default:                                                    // IMP
            if (var_left) return neg ? MK_OP_OR_V : MK_OP_RIMP_V;   // ~x -> A = x | A
            return neg ? MK_OP_IMP_NV : MK_OP_IMP_V;
        }
    }

    // stack holds the first-evaluated operand; swapped: it is the right one
    static int stack_op(Kind k, bool swapped) {
        switch (k) {
        case AND: return MK_OP_AND_S;
        case OR: return MK_OP_OR_S;
        case IFF: return MK_OP_IFF_S;
        default: return swapped ? MK_OP_RIMP_S : MK_OP_IMP_S;    // IMP
        }
    }

    // evaluate node id into A with d stack entries in use
    void gen(int id, int d) {
        if (overflow) return;
        const Node &n = t.nodes[id];
        switch (n.kind) {
        case TOP: emit(MK_OP_LDT, 0); return;
        case BOT: emit(MK_OP_LDF, 0); return;
        case VAR: emit(n.neg ? MK_OP_LDNV : MK_OP_LDV, n.var); return;
        case NOT: gen(n.a, d); emit(MK_OP_NOT, 0); return;
        case BOX: case DIA: {
            const Node &c = t.nodes[n.a];
            if (c.kind == VAR) {            // a modal step on an atom: one instruction
                const bool box = n.kind == BOX;
                emit(box ? (c.neg ? MK_OP_BOX_NV : MK_OP_BOX_V) : (c.neg ? MK_OP_DIA_NV : MK_OP_DIA_V), c.var);
                return;
            }
            gen(n.a, d);
            emit(n.kind == BOX ? MK_OP_BOX : MK_OP_DIA, 0);
            return;
        }
        default: break;
        }
        if (fusable(n)) {
            const bool var_left = !is_var(n.b);
            gen(var_left ? n.b : n.a, d);
            const Node &v = t.nodes[var_left ? n.a : n.b];
            emit(var_op(n.kind, var_left, v.neg), v.var);
            return;
        }
        if (d >= MK_MAX_STACK) { overflow = true; return; }
        const bool left_first = depth(n.a) >= depth(n.b);
        gen(left_first ? n.a : n.b, d);
        emit(MK_OP_PUSH, d);
        if (d + 1 > max_depth) max_depth = d + 1;
        gen(left_first ? n.b : n.a, d + 1);
        emit(stack_op(n.kind, !left_first), d);
    }
};

int compile_tree(Tree &t, int root, int nodes, int depth, int nvars, mk_program *out) {
    // folding can expose new negations (a -> F = ~a) and the normal form new
    // constants (~T = F): two rounds reach the fixed point for every rule here
    int r = fold(t, nnf(t, fold(t, root), false));
    r = fold(t, nnf(t, r, false));
    Gen g(t);
    g.gen(r, 0);
    if (g.overflow) return MK_E_SLOTS;
    if ((int)g.code.size() > MK_MAX_CODE) return MK_E_TOO_LONG;
    std::memset(out, 0, sizeof(*out));
    out->nodes = (uint16_t)nodes;
    out->n_instr = (uint8_t)g.code.size();
    out->nvars = (uint8_t)nvars;
    out->modal_depth = (uint8_t)depth;
    out->depth = (uint8_t)g.max_depth;
    out->n_modal = (uint8_t)g.n_modal;
    out->n_bool = (uint8_t)g.n_bool;
    std::memcpy(out->code, g.code.data(), g.code.size());
    return MK_OK;
}

}  // namespace

extern "C" int mk_compile(const char *text, mk_program *out, int32_t *err_pos) {
    if (err_pos) *err_pos = -1;
    if (!text || !out) return MK_E_ARG;
    Tree t;
    int root = 0;
    Parser p(text, t);
    int rc = p.parse_all(root);
    if (rc != MK_OK) {
        if (err_pos) *err_pos = p.error_pos();
        return rc;
    }
    int nodes = count_nodes(t, root);
    if (nodes > MK_MAX_NODES) return MK_E_TOO_LONG;
    return compile_tree(t, root, nodes, modal_depth(t, root), p.nvars(), out);
}

extern "C" int mk_compile_iff(const char *phi, const char *psi, mk_program *out, int32_t *err_pos) {
    if (err_pos) *err_pos = -1;
    if (!phi || !psi || !out) return MK_E_ARG;
    Tree t;
    int ra = 0, rb = 0;
    Parser pa(phi, t);
    int rc = pa.parse_all(ra);
    if (rc != MK_OK) {
        if (err_pos) *err_pos = pa.error_pos();
        return rc;
    }
    Parser pb(psi, t);
    rc = pb.parse_all(rb);
    if (rc != MK_OK) {
        if (err_pos) *err_pos = pb.error_pos();
        return rc;
    }
    int root = t.add(IFF, ra, rb);
    int nodes = count_nodes(t, root);
    if (nodes > MK_MAX_NODES) return MK_E_TOO_LONG;
    int nv = pa.nvars() > pb.nvars() ? pa.nvars() : pb.nvars();
    return compile_tree(t, root, nodes, modal_depth(t, root), nv, out);
}
