// mk_certify.cpp -- independent certificate checker (host).
//
// Def. 1 / Prop. 2 (Sec. 5): a certificate (phi, n, succ, V, w, C) is valid
// iff the frame belongs to class C and M,w does not satisfy phi.  For a
// separation certificate (Prop. 4) the pointed model must give phi and psi
// different truth values.  The checker is the trust anchor of the search, so
// it shares nothing with the compiler or the kernels: it has its own
// tokenizer and parser, keeps a frame as explicit successor lists, and
// evaluates by the satisfaction clauses of Sec. 2, node by node.
#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "mk.h"

namespace {

struct Formula;
using FormulaPtr = std::shared_ptr<Formula>;

struct Formula {
    enum Op { Top, Bot, Atom, Neg, Conj, Disj, Impl, Bicond, Nec, Poss } op;
    int atom = 0;
    FormulaPtr left, right;
};

FormulaPtr node(Formula::Op op, FormulaPtr l = nullptr, FormulaPtr r = nullptr, int atom = 0) {
    auto f = std::make_shared<Formula>();
    f->op = op;
    f->left = std::move(l);
    f->right = std::move(r);
    f->atom = atom;
    return f;
}

// ---------------------------------------------------------- tokenizer

struct Token {
    enum Kind { End, LParen, RParen, Not, Box, Dia, And, Or, Implies, Iff, True, False, Var, Bad } kind;
    int var = 0;
};

std::vector<Token> tokenize(const std::string &s) {
    std::vector<Token> out;
    size_t i = 0;
    auto word_at = [&](size_t j) { return j < s.size() && (isalnum((unsigned char)s[j]) || s[j] == '_'); };
    while (i < s.size()) {
        char c = s[i];
        if (isspace((unsigned char)c)) { i++; continue; }
        if (s.compare(i, 3, "<->") == 0) { out.push_back({Token::Iff}); i += 3; continue; }
        if (s.compare(i, 2, "->") == 0) { out.push_back({Token::Implies}); i += 2; continue; }
        if (s.compare(i, 2, "[]") == 0) { out.push_back({Token::Box}); i += 2; continue; }
        if (s.compare(i, 2, "<>") == 0) { out.push_back({Token::Dia}); i += 2; continue; }
        if (c == '(') { out.push_back({Token::LParen}); i++; continue; }
        if (c == ')') { out.push_back({Token::RParen}); i++; continue; }
        if (c == '~' || c == '!') { out.push_back({Token::Not}); i++; continue; }
        if (c == '&') { out.push_back({Token::And}); i++; continue; }
        if (c == '|') { out.push_back({Token::Or}); i++; continue; }
        if (isalpha((unsigned char)c)) {
            size_t j = i;
            while (word_at(j)) j++;
            std::string w = s.substr(i, j - i);
            i = j;
            if (w == "not") out.push_back({Token::Not});
            else if (w == "box") out.push_back({Token::Box});
            else if (w == "dia") out.push_back({Token::Dia});
            else if (w == "and") out.push_back({Token::And});
            else if (w == "or") out.push_back({Token::Or});
            else if (w == "T" || w == "true") out.push_back({Token::True});
            else if (w == "F" || w == "false") out.push_back({Token::False});
            else if (w == "p" || w == "q" || w == "r" || w == "s") {
                Token t{Token::Var};
                t.var = std::string("pqrs").find(w[0]);
                out.push_back(t);
            } else if (w.size() >= 2 && w[0] == 'p' && w.find_first_not_of("0123456789", 1) == std::string::npos
                       && w.size() <= 4) {
                Token t{Token::Var};
                t.var = std::stoi(w.substr(1));
                out.push_back(t);
            } else {
                out.push_back({Token::Bad});
            }
            continue;
        }
        out.push_back({Token::Bad});
        i++;
    }
    out.push_back({Token::End});
    return out;
}

// ------------------------------------------------------------- parser

class Reader {
  public:
    explicit Reader(std::vector<Token> t) : toks_(std::move(t)) {}
    FormulaPtr formula() {
        FormulaPtr f = bicond();
        if (toks_[pos_].kind != Token::End) ok_ = false;
        return ok_ ? f : nullptr;
    }
    int max_var() const { return max_var_; }

  private:
    std::vector<Token> toks_;
    size_t pos_ = 0;
    bool ok_ = true;
    int max_var_ = -1;

    Token::Kind peek() const { return toks_[pos_].kind; }
    bool accept(Token::Kind k) {
        if (peek() != k) return false;
        pos_++;
        return true;
    }
    FormulaPtr bicond() {
        FormulaPtr f = implication();
        while (ok_ && accept(Token::Iff)) f = node(Formula::Bicond, f, implication());
        return f;
    }
    FormulaPtr implication() {
        FormulaPtr f = disjunction();
        if (ok_ && accept(Token::Implies)) return node(Formula::Impl, f, implication());
        return f;
    }
    FormulaPtr disjunction() {
        FormulaPtr f = conjunction();
        while (ok_ && accept(Token::Or)) f = node(Formula::Disj, f, conjunction());
        return f;
    }
    FormulaPtr conjunction() {
        FormulaPtr f = prefix();
        while (ok_ && accept(Token::And)) f = node(Formula::Conj, f, prefix());
        return f;
    }
    FormulaPtr prefix() {
        if (!ok_) return nullptr;
        if (accept(Token::Not)) return node(Formula::Neg, prefix());
        if (accept(Token::Box)) return node(Formula::Nec, prefix());
        if (accept(Token::Dia)) return node(Formula::Poss, prefix());
        if (accept(Token::True)) return node(Formula::Top);
        if (accept(Token::False)) return node(Formula::Bot);
        if (peek() == Token::Var) {
            int v = toks_[pos_++].var;
            if (v > max_var_) max_var_ = v;
            return node(Formula::Atom, nullptr, nullptr, v);
        }
        if (accept(Token::LParen)) {
            FormulaPtr f = bicond();
            if (!accept(Token::RParen)) ok_ = false;
            return f;
        }
        ok_ = false;
        return nullptr;
    }
};

// ------------------------------------------------------ explicit models

struct Model {
    int n;
    std::vector<std::vector<int>> successors;   // successors[w] = {v : R(w,v)}
    std::vector<std::vector<bool>> atom_true;   // atom_true[i][w]
};

bool related(const Model &m, int w, int v) {
    for (int u : m.successors[w]) if (u == v) return true;
    return false;
}

// the set of worlds where f holds, by the clauses of Sec. 2
std::vector<bool> holds(const Model &m, const Formula &f) {
    std::vector<bool> out(m.n, false);
    switch (f.op) {
    case Formula::Top: out.assign(m.n, true); break;
    case Formula::Bot: break;
    case Formula::Atom:
        if (f.atom < (int)m.atom_true.size()) out = m.atom_true[f.atom];
        break;
    case Formula::Neg: {
        auto a = holds(m, *f.left);
        for (int w = 0; w < m.n; w++) out[w] = !a[w];
        break;
    }
    case Formula::Conj: case Formula::Disj: case Formula::Impl: case Formula::Bicond: {
        auto a = holds(m, *f.left), b = holds(m, *f.right);
        for (int w = 0; w < m.n; w++) {
            if (f.op == Formula::Conj) out[w] = a[w] && b[w];
            else if (f.op == Formula::Disj) out[w] = a[w] || b[w];
            else if (f.op == Formula::Impl) out[w] = !a[w] || b[w];
            else out[w] = a[w] == b[w];
        }
        break;
    }
    case Formula::Nec: {       // true at w iff every successor satisfies the argument
        auto a = holds(m, *f.left);
        for (int w = 0; w < m.n; w++) {
            bool all = true;
            for (int v : m.successors[w]) all = all && a[v];
            out[w] = all;
        }
        break;
    }
    case Formula::Poss: {      // true at w iff some successor satisfies the argument
        auto a = holds(m, *f.left);
        for (int w = 0; w < m.n; w++) {
            bool any = false;
            for (int v : m.successors[w]) any = any || a[v];
            out[w] = any;
        }
        break;
    }
    }
    return out;
}

bool frame_in_class(const Model &m, int cls) {
    if (cls == 0) return true;
    if (cls == 4) {                                                             // K4: transitive
        for (int w = 0; w < m.n; w++)
            for (int v : m.successors[w])
                for (int u : m.successors[v])
                    if (!related(m, w, u)) return false;
        return true;
    }
    for (int w = 0; w < m.n; w++) if (!related(m, w, w)) return false;          // reflexive
    if (cls == 1) return true;
    for (int w = 0; w < m.n; w++)                                               // transitive
        for (int v : m.successors[w])
            for (int u : m.successors[v])
                if (!related(m, w, u)) return false;
    if (cls == 2) return true;
    for (int w = 0; w < m.n; w++)                                               // symmetric
        for (int v : m.successors[w])
            if (!related(m, v, w)) return false;
    return true;
}

}  // namespace

extern "C" int mk_certify(const mk_cert *c) {
    if (!c || !c->phi) return MK_E_ARG;
    int n = c->n;
    if (n < 1 || n > MK_MAX_CERT_WORLDS || c->cls > 4 || c->world >= n) return MK_E_ARG;
    uint64_t full = (n == 32) ? 0xFFFFFFFFull : ((1ull << n) - 1);
    Reader ra(tokenize(c->phi));
    FormulaPtr phi = ra.formula();
    if (!phi) return MK_E_SYNTAX;
    FormulaPtr psi;
    int max_var = ra.max_var();
    if (c->psi) {
        Reader rb(tokenize(c->psi));
        psi = rb.formula();
        if (!psi) return MK_E_SYNTAX;
        if (rb.max_var() > max_var) max_var = rb.max_var();
    }
    if (max_var >= MK_MAX_VARS) return MK_E_VARS;

    Model m;
    m.n = n;
    m.successors.assign(n, {});
    for (int w = 0; w < n; w++) {
        if ((uint64_t)c->succ[w] & ~full) return MK_E_ARG;
        for (int v = 0; v < n; v++)
            if ((c->succ[w] >> v) & 1u) m.successors[w].push_back(v);
    }
    m.atom_true.assign(MK_MAX_VARS, std::vector<bool>(n, false));
    for (int i = 0; i < MK_MAX_VARS; i++) {
        if ((uint64_t)c->val[i] & ~full) return MK_E_ARG;
        for (int w = 0; w < n; w++) m.atom_true[i][w] = (c->val[i] >> w) & 1u;
    }
    if (!frame_in_class(m, c->cls)) return 0;
    bool a = holds(m, *phi)[c->world];
    if (!psi) return a ? 0 : 1;
    bool b = holds(m, *psi)[c->world];
    return a != b ? 1 : 0;
}
