"""The pins of the oracle's Python code (GLL rule, network, unique-node vectors, the dense brute-force
operator) catch plausible mistakes.

Each case plants one mistake (a wrong power, a flipped sign, swapped indices, a dropped term, a shift the wrong
way, an overwrite in place of a sum) in a copy of a module's source, executes the copy, puts its functions in
place of the module's for the duration of the check, and checks that a pin fails under it.  The committed
oracle is never modified.
"""
import numpy as np
import pytest

from oracle import gll, lvec, net, ref
from tests import test_oracle_ax as tax
from tests import test_oracle_gll as tg
from tests import test_oracle_lvec as tl
from tests import test_oracle_net as tn

MUTANTS = [
    # GLL rule: weights 2 / (N (N+1) L_N(x)^2), corner entries of D -+N(N+1)/4,
    # off-diagonal entries L_N(x_i) / (L_N(x_l) (x_i - x_l))
    ("gll_weight_power", gll, "rho = 2.0 / (N * (N + 1) * LN ** 2)", "rho = 2.0 / (N * (N + 1) * LN)",
     lambda: tg.test_quadrature_exact_to_degree_2N_minus_1(5)),
    ("gll_corner_sign", gll, "D[0, 0] = -N * (N + 1) / 4.0", "D[0, 0] = N * (N + 1) / 4.0",
     lambda: tg.test_derivative_of_monomials(5)),
    ("gll_offdiagonal_ratio_swapped", gll, "D[i, l] = LN[i] / (LN[l] * (xi[i] - xi[l]))",
     "D[i, l] = LN[l] / (LN[i] * (xi[i] - xi[l]))", lambda: tg.test_D_is_lagrange_derivative_by_brute_force(6)),
    # network: convolution taps, GELU derivative, backward pass, Adam
    ("conv_shift_wrong_way", net, 'y += np.einsum("oc,bckji->bokji", W[:, :, t], shift(x, dk, dj, di))',
     'y += np.einsum("oc,bckji->bokji", W[:, :, t], shift(x, -dk, -dj, -di))', tn.test_conv_matches_loop_definition),
    ("gelu_grad_density_term_dropped", net,
     "return 0.5 * (1.0 + erf(v / math.sqrt(2.0))) + v * np.exp(-0.5 * v * v) / math.sqrt(2.0 * math.pi)",
     "return 0.5 * (1.0 + erf(v / math.sqrt(2.0)))", tn.test_gelu_values_and_derivative),
    ("backward_activation_for_preactivation", net, 'dh2 = conv_input_grad(dy, P["W3"]) * gelu_grad(h2)',
     'dh2 = conv_input_grad(dy, P["W3"]) * gelu_grad(a2)', lambda: tn.test_gradients_by_central_differences(3)),
    ("weight_grad_shift_wrong_way", net, 'dW[:, :, t] = np.einsum("bokji,bckji->oc", dy, shift(x, dk, dj, di))',
     'dW[:, :, t] = np.einsum("bokji,bckji->oc", dy, shift(x, -dk, -dj, -di))',
     lambda: tn.test_gradients_by_central_differences(3)),
    ("adam_second_moment_bias_uses_b1", net, "vh = v / (1 - b2 ** t)", "vh = v / (1 - b1 ** t)",
     tn.test_adam_matches_scalar_recurrence),
    # unique-node vectors: Q^T sums the copies; PCG's beta
    ("assemble_overwrites_copies", lvec,
     "return np.bincount(np.asarray(l2g).reshape(-1), weights=np.asarray(w, dtype=np.float64).reshape(-1),\n"
     "                       minlength=nL)",
     "out = np.zeros(nL)\n    out[np.asarray(l2g).reshape(-1)] = np.asarray(w, dtype=np.float64).reshape(-1)\n"
     "    return out", lambda: tl.test_apply_equals_dense_assembled_matrix((2, 2, 1), 3)),
    ("lvec_cg_beta_inverted", lvec, "beta = rz_new / rz", "beta = rz / rz_new",
     lambda: tl.test_same_iterates_as_the_element_vector_solve((3, 2, 2), 4)),
    # the dense brute-force operator (itself a pin of the C operator): Kronecker factor order, G components
    ("dense_s_gradient_kron_order", ref, "Bs = np.kron(I, np.kron(D, I))", "Bs = np.kron(D, np.kron(I, I))",
     lambda: tax.test_dense_brute_force(3)),
    ("dense_offdiagonal_components_swapped", ref, "(0, 1): 1, (0, 2): 2", "(0, 1): 2, (0, 2): 1",
     lambda: tax.test_dense_brute_force(3)),
]


@pytest.mark.parametrize("name,mod,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_python_pin_catches_planted_mistake(name, mod, old, new, check, monkeypatch):
    path = mod.__file__
    with open(path) as fh:
        src = fh.read()
    assert src.count(old) == 1, name
    check()  # the unmodified oracle passes the pin
    ns = {"__name__": mod.__name__ + "_mutant", "__package__": "oracle", "__file__": path}
    exec(compile(src.replace(old, new), path, "exec"), ns)
    swapped = 0
    for k, v in list(ns.items()):
        if callable(v) and getattr(v, "__module__", None) == ns["__name__"] and hasattr(mod, k):
            monkeypatch.setattr(mod, k, v)
            swapped += 1
    assert swapped > 0
    with np.errstate(all="ignore"):
        with pytest.raises((AssertionError, np.linalg.LinAlgError, ValueError, ZeroDivisionError)):
            check()
