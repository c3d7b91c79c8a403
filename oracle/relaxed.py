"""FP64 reference of the relaxed (differentiable) fixpoint -- test infrastructure only.

The paper defines the exact operator theta(M_P v) (Def. 2, Def. 5, Algorithm 1). The relaxed
path replaces the step threshold by a sigmoid of temperature tau and gives every rule row a
weight, so that the unrolled iteration is differentiable; the hardened limit (tau -> 0, binary
inputs) is the exact iteration. Row by row, with x = (M_P v)_i the paper's row sum:

    rule row of rule r, m body atoms (entries 1/m):  u_i = sigmoid(w_r * (x - 1 + 1/(2m)) / tau)
    OR-rule row (entries 1):                          u_i = sigmoid((x - 1/2) / tau)
    self-loop (fact, barred atom: a_ii = 1):          u_i = v_i
    empty row:                                        u_i = 0

With binary v, a rule row's x is 1 when all m atoms hold and at most 1 - 1/m otherwise, so the
logit is >= w/(2m tau) or <= -w/(2m tau); an OR row's x is >= 1 or 0, so the logit is >= 1/(2 tau)
or -1/(2 tau): the hardened rows are theta exactly.

Reverse mode (written out): with g = dL/dv_{t+1} and e_i = g_i u_i (1 - u_i),
    dL/dw_r += sum over the batch of e_i (x_i - 1 + 1/(2m)) / tau           (rule rows)
    dL/dv_t  = M_P^T (c * e) + g on self-loop rows,  c_i = w_r / tau (rule), 1 / tau (OR)
(the entries of M_P carry the 1/m). Everything is float64 (numpy + scipy.sparse).
"""
import numpy as np
import scipy.sparse as sp

from . import ORC_AND, ORC_BARRED, ORC_EMPTY, ORC_FACT, ORC_OR, standardize


class RelaxedProgram:
    """Standardized matrix (canonical order) plus the rule of every rule row."""

    def __init__(self, prog, std=None):
        self.std = std or standardize(prog)
        s = self.std
        self.n_prime = s.n_prime
        rows = np.repeat(np.arange(s.n_prime), np.diff(s.row_ptr))
        vals = s.num.astype(np.float64) / s.den[rows].astype(np.float64)
        self.M = sp.csr_matrix((vals, (rows, s.col)), shape=(s.n_prime, s.n_prime))
        self.kind = s.kind.copy()
        self.m = np.diff(s.row_ptr).astype(np.float64)
        # the original rule behind each rule row (standardization of Sec. 2.1): a head with one
        # rule keeps it in its own row; a head with several rules gets one new atom per rule,
        # numbered after the originals and barred atoms in rule order
        head = np.asarray(prog.head, dtype=np.int64)
        n, nr = int(prog.n_atoms), len(head)
        cnt = np.bincount(head, minlength=n)
        rule_of_row = np.full(s.n_prime, -1, dtype=np.int64)
        single = cnt[head] == 1
        rule_of_row[head[single]] = np.nonzero(single)[0]
        multi = np.nonzero(~single)[0]
        rule_of_row[n + s.n_barred + np.arange(len(multi))] = multi
        rule_of_row[self.kind != ORC_AND] = -1
        self.rule_of_row = rule_of_row
        self.n_rules = nr
        self.is_rule = self.kind == ORC_AND
        self.is_or = self.kind == ORC_OR
        self.is_self = (self.kind == ORC_FACT) | (self.kind == ORC_BARRED)
        self.is_empty = self.kind == ORC_EMPTY

    def row_weights(self, w):
        wr = np.zeros(self.n_prime)
        wr[self.is_rule] = np.asarray(w, dtype=np.float64)[self.rule_of_row[self.is_rule]]
        return wr

    def step(self, v, wr, tau):
        """One relaxed application; v is (n', b). Returns (u, x) with x = M_P v."""
        x = self.M @ v
        u = np.zeros_like(v)
        r, o = self.is_rule, self.is_or
        u[r] = _sigmoid(wr[r, None] * (x[r] - 1.0 + 1.0 / (2.0 * self.m[r, None])) / tau)
        u[o] = _sigmoid((x[o] - 0.5) / tau)
        u[self.is_self] = v[self.is_self]
        return u, x

    def forward(self, w, v0, T, tau):
        """v_0 .. v_T (list of (n', b) arrays)."""
        wr = self.row_weights(w)
        vs = [np.asarray(v0, dtype=np.float64)]
        for _ in range(T):
            vs.append(self.step(vs[-1], wr, tau)[0])
        return vs

    def backward(self, w, vs, gT, tau):
        """Reverse mode through v_0 .. v_T; returns (dL/dw per original rule, dL/dv_0)."""
        wr = self.row_weights(w)
        r, o, sf = self.is_rule, self.is_or, self.is_self
        dwr = np.zeros(self.n_prime)
        g = np.asarray(gT, dtype=np.float64)
        MT = self.M.T.tocsr()
        for t in range(len(vs) - 2, -1, -1):
            u, x = self.step(vs[t], wr, tau)
            e = np.zeros_like(g)
            e[r | o] = g[r | o] * u[r | o] * (1.0 - u[r | o])
            dwr[r] += np.sum(e[r] * (x[r] - 1.0 + 1.0 / (2.0 * self.m[r, None])), axis=1) / tau
            c = np.zeros(self.n_prime)
            c[r] = wr[r] / tau
            c[o] = 1.0 / tau
            gp = MT @ (c[:, None] * e)
            gp[sf] += g[sf]
            g = gp
        dw = np.zeros(self.n_rules)
        dw[self.rule_of_row[r]] = dwr[r]
        return dw, g


def _sigmoid(z):
    return 0.5 * (1.0 + np.tanh(0.5 * z))  # stable for large |z|
