"""Error measures (oracle side; test infrastructure).

* ``rel_pred_error`` - ||X(beta - beta-hat)|| / ||X beta-hat||, the relative
  OLS prediction error used to judge every solve against the OLS estimator.
* ``delta_t`` - the paper's accuracy measure Delta_t = ||X(beta_t - beta)||^2
  against the true parameter (Sec. 4); the OLS level is sigma^2 d.
"""
import numpy as np


def rel_pred_error(X, beta, beta_hat):
    diff = np.asarray(X) @ (np.asarray(beta) - np.asarray(beta_hat))
    return float(np.linalg.norm(diff) / np.linalg.norm(np.asarray(X) @ beta_hat))


def delta_t(X, beta_t, beta_true):
    diff = np.asarray(X) @ (np.asarray(beta_t) - np.asarray(beta_true))
    return float(diff @ diff)
