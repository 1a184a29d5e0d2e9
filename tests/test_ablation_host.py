"""Host logic of the control-parameter studies: NSE budgets and the settings they run."""
from paper_2107_09801_gb300.ablation import Setting, SettingResult, moves_for_nse


def test_nse_budget_counts_one_evaluation_per_window_neighbour():
    assert moves_for_nse(10**10, 65535) == -(-10**10 // 6912)     # the paper's runs: 1 446 760 moves
    assert moves_for_nse(6912, 65535) == 1
    assert moves_for_nse(6913, 65535) == 2
    assert moves_for_nse(1000, 255) == 4                           # N = L when L < N_lmt
    assert moves_for_nse(1, 255) == 1


def test_setting_result_statistics():
    r = SettingResult(Setting(4, 13, 2000, 10), [212, 214, 213])
    assert r.mean == 213.0 and abs(r.std - 1.0) < 1e-12
    assert SettingResult(Setting(4, 4, 2000, 10), [7]).std == 0.0
